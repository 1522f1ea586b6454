// sv_api.cu -- the C ABI (include/stokes_vanka.h): hierarchy set-up, the
// V-cycle of Algorithm 1 driven from the host as a sequence of stream-ordered
// kernel launches, and right-preconditioned FGMRES (Section 6.8) with every
// vector operation on the device.  Only scalars of the convergence test cross
// to the host (one 8-byte copy per iteration).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sv_internal.h"

namespace {

thread_local std::string g_err;

stokes_status fail(stokes_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

stokes_status cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define SV_TRY(call, where)                       \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

stokes_status check_launch(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, where);
  return STOKES_OK;
}

struct UnitSchur {
  double z[50];
  double s;
};

const UnitSchur& unit_schur() {
  static const UnitSchur u = [] {
    UnitSchur v{};
    sv::interior_unit_schur(v.z, &v.s);
    return v;
  }();
  return u;
}

sv::LevelDev make_level(int n, double nu) {
  sv::LevelDev d;
  d.n = n;
  d.nq = 2 * n + 1;
  d.np = n + 1;
  d.nv = static_cast<long long>(d.nq) * d.nq;
  d.N = 2 * d.nv + static_cast<long long>(d.np) * d.np;
  d.h = 1.0 / n;
  d.nu = nu;
  d.cl = nu / 90.0;
  d.cb = -d.h / 18.0;
  d.clf = static_cast<float>(d.cl);
  d.cbf = static_cast<float>(d.cb);
  d.zs = d.cb / d.cl;
  d.zsinv = 1.0 / (d.cb * d.zs * unit_schur().s);
  d.zsf = static_cast<float>(d.zs);
  d.zsinvf = static_cast<float>(d.zsinv);
  return d;
}

void free_all(stokes_hierarchy* h) {
  for (auto& L : h->lv) {
    cudaFree(L.x0);
    cudaFree(L.x1);
    cudaFree(L.b);
    cudaFree(L.r);
    cudaFree(L.e);
    cudaFree(L.cd);
    cudaFree(L.xf0);
    cudaFree(L.xf1);
    cudaFree(L.bf);
    cudaFree(L.rf);
    cudaFree(L.ef);
    cudaFree(L.cdf);
    cudaFree(L.tcB);
    cudaFree(L.pinv);
  }
  cudaFree(h->delta);
  h->delta = nullptr;
  cudaFree(h->deltaf);
  h->deltaf = nullptr;
  cudaFree(h->bs_buf);
  h->bs_buf = nullptr;
  cudaFree(h->bt_GL);
  cudaFree(h->bt_GM);
  cudaFree(h->bt_buf);
  h->bt_GL = h->bt_GM = h->bt_buf = nullptr;
  h->lv.clear();
  cudaFree(h->coarse_G);
  cudaFree(h->V);
  cudaFree(h->Z);
  cudaFree(h->small);
  cudaFree(h->partials);
  cudaFree(h->dev_err);
  h->dev_err = nullptr;
  cudaFree(h->ticket);
  h->ticket = nullptr;
  cudaFree(h->aux);
  h->aux = nullptr;
  cudaFree(h->tail_ops);
  cudaFree(h->tail_levels);
  cudaFree(h->tail_bar);
  h->tail_ops = nullptr;
  h->tail_levels = nullptr;
  h->tail_bar = nullptr;
  h->tail_top = -1;
  if (h->ring_stream) {
    cudaStreamSynchronize(h->ring_stream);
    cudaStreamDestroy(h->ring_stream);
  }
  if (h->ring_fork) cudaEventDestroy(h->ring_fork);
  if (h->ring_join) cudaEventDestroy(h->ring_join);
  h->ring_stream = nullptr;
  h->ring_fork = h->ring_join = nullptr;
  if (h->host_scalars) cudaFreeHost(h->host_scalars);
  h->coarse_G = h->V = h->Z = h->small = h->partials = h->host_scalars = nullptr;
}

// Device allocations of stokes_hierarchy_create go through dalloc.  A test hook
// (stokes_test_set_alloc_limit) caps the bytes one creation may allocate, so the
// STOKES_ERR_OOM path runs without exhausting the GPU.
std::atomic<long long> g_alloc_cap{0};      // 0: no cap
thread_local long long t_alloc_used = 0;    // bytes allocated by the creation running on this thread

cudaError_t dalloc_bytes(void** p, size_t bytes) {
  const long long cap = g_alloc_cap.load();
  if (cap > 0 && t_alloc_used + static_cast<long long>(bytes) > cap) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) t_alloc_used += static_cast<long long>(bytes);
  return e;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return dalloc_bytes(reinterpret_cast<void**>(p), count * sizeof(T));
}

stokes_status check_level(const stokes_hierarchy* h, int level, int min_level = 0) {
  if (h == nullptr) return fail(STOKES_ERR_ARG, "null hierarchy");
  if (level < min_level || level >= static_cast<int>(h->lv.size()))
    return fail(STOKES_ERR_ARG, "level index out of range");
  return STOKES_OK;
}

// Launch one sweep; on the finest level, bracket it with a CUDA-event pair
// when timing is on (events are pooled and summed in stokes_stats_read).
template <typename R>
void timed_sweep(stokes_hierarchy* h, bool finest, sv::Level& L, const R* x, const R* b, R* xo);

cudaEvent_t* timing_pair(stokes_hierarchy* h, bool finest) {
  if (!(h->timing && finest)) return nullptr;
  if (h->ev_used + 2 > h->ev_pool.size()) {
    for (int k = 0; k < 64; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) break;
      h->ev_pool.push_back(e);
    }
  }
  if (h->ev_used + 2 > h->ev_pool.size()) return nullptr;
  cudaEvent_t* p = &h->ev_pool[h->ev_used];
  h->ev_used += 2;
  return p;
}

// One FP64 sweep with the hierarchy's smoother (shared class factors, or the
// stored per-patch inverses, whose sweep uses L.r as residual scratch: L.r is
// free whenever a sweep runs).
void sweep_f64(stokes_hierarchy* h, sv::Level& L, const double* x, const double* b, double* xo) {
  if (h->prm.smoother == STOKES_SMOOTHER_BRAESS_SARAZIN || h->prm.smoother == STOKES_SMOOTHER_SCHUR_UZAWA)
    sv::launch_bs_sweep<double>(L.d, h->bs, static_cast<double*>(h->bs_buf), L.r, x, b, xo, h->stream);
  else if (h->prm.smoother == STOKES_SMOOTHER_PER_PATCH)
    sv::launch_simple_sweep(L.d, L.pinv, h->delta, L.r, x, b, xo, h->prm.omega, h->stream);
  else if (sv::vanka_cfg_split(L.vk_cfg))
    sv::launch_vanka_split<double>(L.d, L.cd, h->fd, x, b, xo, h->prm.omega, h->delta, L.vk_cfg == sv::VANKA_CFG_SPLIT2,
                           h->stream, L.r);
  else
    sv::launch_vanka<double>(L.d, L.cd, h->fd, x, b, xo, h->prm.omega, L.vk_cfg, h->stream);
}

// Mixed-form sweep of a level with strip tiles: the interior tiles on the strip
// kernel (stream s) -- the tensor-core GEMM in the BF16 form, the FP32 fast-
// diagonalisation solve in the FP32 form -- and the ring of boundary tiles on the
// SIMT kernel (ring_stream), concurrently: both read x and b and write disjoint
// owned dofs of xo.  Fork and join are event waits, valid eagerly and under capture.
void tc_sweep(stokes_hierarchy* h, sv::Level& L, const float* x, const float* b, float* xo, cudaStream_t s) {
  cudaEventRecord(h->ring_fork, s);
  cudaStreamWaitEvent(h->ring_stream, h->ring_fork, 0);
  sv::launch_vanka<float>(L.d, L.cdf, h->fdf, x, b, xo, h->prm.omega, sv::VANKA_CFG_14, h->ring_stream, L.tc_lo,
                          L.tc_hi);
  if (h->prm.prec == STOKES_MIXED_BF16)
    sv::launch_vanka_tc(L.d, L.tcB, x, b, xo, h->prm.omega, L.tc_lo, L.tc_hi, h->dev_err, s, h->tc_wait_limit);
  else
    sv::launch_vanka_strip_f32(L.d, h->fdf, x, b, xo, h->prm.omega, L.tc_lo, L.tc_hi, s);
  cudaEventRecord(h->ring_join, h->ring_stream);
  cudaStreamWaitEvent(s, h->ring_join, 0);
}

template <>
void timed_sweep<double>(stokes_hierarchy* h, bool finest, sv::Level& L, const double* x, const double* b,
                         double* xo) {
  cudaEvent_t* ev = timing_pair(h, finest);
  if (ev) cudaEventRecord(ev[0], h->stream);
  sweep_f64(h, L, x, b, xo);
  if (ev) cudaEventRecord(ev[1], h->stream);
}

template <>
void timed_sweep<float>(stokes_hierarchy* h, bool finest, sv::Level& L, const float* x, const float* b,
                        float* xo) {
  cudaEvent_t* ev = timing_pair(h, finest);
  if (ev) cudaEventRecord(ev[0], h->stream);
  if (h->prm.smoother == STOKES_SMOOTHER_BRAESS_SARAZIN || h->prm.smoother == STOKES_SMOOTHER_SCHUR_UZAWA) {
    sv::launch_bs_sweep<float>(L.d, h->bs, static_cast<float*>(h->bs_buf), L.rf, x, b, xo, h->stream);
  } else if (L.strip && L.tc_on) {
    tc_sweep(h, L, x, b, xo, h->stream);
  } else if (sv::vanka_cfg_split(L.vk_cfg_f)) {
    sv::launch_vanka_split<float>(L.d, L.cdf, h->fdf, x, b, xo, h->prm.omega, h->deltaf,
                                  L.vk_cfg_f == sv::VANKA_CFG_SPLIT2, h->stream, nullptr);
  } else {
    sv::launch_vanka<float>(L.d, L.cdf, h->fdf, x, b, xo, h->prm.omega, L.vk_cfg_f, h->stream);
  }
  if (ev) cudaEventRecord(ev[1], h->stream);
}

// ---- V-cycle (Algorithm 1) ----
// Level buffers of the precision R: the FP64 set (x0, x1, b, r, e) or the
// FP32 set of the mixed-precision preconditioner (xf0, xf1, bf, rf, ef).
template <typename R>
struct Buf;
template <>
struct Buf<double> {
  static double* x0(sv::Level& L) { return L.x0; }
  static double* x1(sv::Level& L) { return L.x1; }
  static double* b(sv::Level& L) { return L.b; }
  static double* r(sv::Level& L) { return L.r; }
  static double* e(sv::Level& L) { return L.e; }
};
template <>
struct Buf<float> {
  static float* x0(sv::Level& L) { return L.xf0; }
  static float* x1(sv::Level& L) { return L.xf1; }
  static float* b(sv::Level& L) { return L.bf; }
  static float* r(sv::Level& L) { return L.rf; }
  static float* e(sv::Level& L) { return L.ef; }
};

// Exact coarse solve in FP64 (Algorithm 1, level 0), for either precision.
void coarse_apply(stokes_hierarchy* h, const double* b, double* out) {
  sv::launch_coarse(h->coarse_G, h->N0, b, out, h->stream);
}
void coarse_apply(stokes_hierarchy* h, const float* b, float* out) {
  sv::Level& C = h->lv[0];
  sv::launch_convert<float, double>(b, C.b, C.d.N, h->stream);
  sv::launch_coarse(h->coarse_G, h->N0, C.b, C.e, h->stream);
  sv::launch_convert<double, float>(C.e, out, C.d.N, h->stream);
}

// NVTX range names of the levels (host-side markers for profilers; free when no
// tool is attached): "mg level <l> n=<n>"
const char* level_range_name(const sv::Level& L, int l) {
  static thread_local char buf[48];
  std::snprintf(buf, sizeof(buf), "mg level %d n=%d", l, L.d.n);
  return buf;
}

template <typename R>
void vcycle_level(stokes_hierarchy* h, int l, const R* b, R* out);

// The persistent coarse-level launch (FP32 cycles only): levels 0..tail_top in one
// cooperative kernel running the steps recorded by tail_build.
bool run_tail(stokes_hierarchy* h, int l, const double*, double*) { (void)h; (void)l; return false; }
bool run_tail(stokes_hierarchy* h, int l, const float* b, float* out) {
  if (l != h->tail_top || b != h->lv[l].bf || out != h->lv[l].ef) return false;
  nvtxRangePushA("mg levels 0..tail (persistent launch)");
  if (h->prm.tail_n > 0) {
    sv::launch_tail(h->tail_ops, h->tail_nops, h->tail_levels, h->coarse_G, h->N0, h->fdf, h->prm.omega,
                    h->tail_bar, h->dev_err, h->tail_spin_limit, h->tail_skip_arrival, h->tail_grid, h->stream);
  } else {   // test mode: the same kernel and steps, one launch per step (no grid barrier)
    for (int k = 0; k < h->tail_nops; ++k)
      sv::launch_tail(h->tail_ops + k, 1, h->tail_levels, h->coarse_G, h->N0, h->fdf, h->prm.omega, h->tail_bar,
                      h->dev_err, h->tail_spin_limit, -1, h->tail_grid, h->stream);
  }
  nvtxRangePop();
  return true;
}

template <typename R>
void vcycle(stokes_hierarchy* h, int l, const R* b, R* out) {
  if (run_tail(h, l, b, out)) return;
  nvtxRangePushA(level_range_name(h->lv[l], l));
  vcycle_level<R>(h, l, b, out);
  nvtxRangePop();
}

// The steps of vcycle_level<float> on level l and below, in launch order, with the
// same buffers (Algorithm 1; the coarse solve through the bordered inverse).
void tail_build(stokes_hierarchy* h, int l, const float* b, float* out, std::vector<sv::TailOp>& ops) {
  sv::Level& L = h->lv[l];
  if (l == 0) {
    ops.push_back({sv::TAIL_COARSE, 0, b, nullptr, out});
    return;
  }
  float* X0 = L.xf0;
  float* X1 = L.xf1;
  float* cur = nullptr;
  for (int it = 0; it < h->prm.nu1; ++it) {
    float* dst = (cur == X0) ? X1 : X0;
    ops.push_back({sv::TAIL_SWEEP, l, cur, b, dst});
    cur = dst;
  }
  if (cur == nullptr) {
    ops.push_back({sv::TAIL_ZERO, l, nullptr, nullptr, X0});
    cur = X0;
  }
  sv::Level& C = h->lv[l - 1];
  const int passes = (l - 1 == 0) ? 1 : h->prm.cycle;
  for (int g = 0; g < passes; ++g) {
    ops.push_back({sv::TAIL_RESID, l, cur, b, L.rf});
    ops.push_back({sv::TAIL_RESTRICT, l, L.rf, nullptr, C.bf});
    tail_build(h, l - 1, C.bf, C.ef, ops);
    ops.push_back({sv::TAIL_PROLONG, l, C.ef, nullptr, cur});
  }
  for (int it = 0; it < h->prm.nu2; ++it) {
    float* dst = (it == h->prm.nu2 - 1) ? out : ((cur == X0) ? X1 : X0);
    ops.push_back({sv::TAIL_SWEEP, l, cur, b, dst});
    cur = dst;
  }
  if (h->prm.nu2 == 0) ops.push_back({sv::TAIL_COPY, l, cur, nullptr, out});
}

// Levels n <= tail_n below the finest one, for an FP32 Vanka cycle: the tail's
// step list, level table and barrier state on the device.
cudaError_t tail_setup(stokes_hierarchy* h) {
  const int top = static_cast<int>(h->lv.size()) - 2;
  const int tail_n = h->prm.tail_n < 0 ? -h->prm.tail_n : h->prm.tail_n;
  if (tail_n == 0 || h->prm.prec == STOKES_FP64 || h->prm.smoother != STOKES_SMOOTHER_SHARED ||
      h->prm.precond != 0 || top < 1)
    return cudaSuccess;
  int t = -1;
  for (int l = 1; l <= top; ++l)
    if (h->lv[l].d.n <= tail_n) t = l;
  if (t < 1 || t > 7) return cudaSuccess;
  int max_ctas = 0;
  cudaError_t e = sv::tail_prepare(&max_ctas);
  if (e != cudaSuccess) return e;
  std::vector<sv::TailOp> ops;
  tail_build(h, t, h->lv[t].bf, h->lv[t].ef, ops);
  std::vector<sv::TailLevel> lv(t + 1);
  for (int l = 0; l <= t; ++l) lv[l] = {h->lv[l].d, h->lv[l].cdf};
  const int np = h->lv[t].d.np, tiles = ((np + 7) / 8) * ((np + 7) / 8);
  h->tail_grid = max_ctas < tiles ? max_ctas : tiles;
  if (h->tail_grid < 1) return cudaSuccess;
  if ((e = dalloc(&h->tail_ops, ops.size())) != cudaSuccess) return e;
  if ((e = dalloc(&h->tail_levels, lv.size())) != cudaSuccess) return e;
  if ((e = dalloc(&h->tail_bar, 2)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(h->tail_ops, ops.data(), ops.size() * sizeof(sv::TailOp), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpy(h->tail_levels, lv.data(), lv.size() * sizeof(sv::TailLevel), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemset(h->tail_bar, 0, 2 * sizeof(unsigned))) != cudaSuccess) return e;
  h->tail_nops = static_cast<int>(ops.size());
  h->tail_top = t;
  return cudaSuccess;
}

template <typename R>
void vcycle_level(stokes_hierarchy* h, int l, const R* b, R* out) {
  cudaStream_t s = h->stream;
  sv::Level& L = h->lv[l];
  if (l == 0) {
    coarse_apply(h, b, out);
    return;
  }
  const bool finest = (l == static_cast<int>(h->lv.size()) - 1);
  R* X0 = Buf<R>::x0(L);
  R* X1 = Buf<R>::x1(L);
  R* cur = nullptr;  // nullptr = zero initial guess
  for (int it = 0; it < h->prm.nu1; ++it) {
    R* dst = (cur == X0) ? X1 : X0;
    timed_sweep<R>(h, finest, L, cur, b, dst);
    cur = dst;
  }
  if (cur == nullptr) {
    cudaMemsetAsync(X0, 0, L.d.N * sizeof(R), s);
    cur = X0;
  }
  sv::Level& C = h->lv[l - 1];
  // coarse-grid correction, cycle times (W-cycle: 2) below the coarsest-but-one level;
  // restricting the updated fine residual gives the coarse residual r_c - A_c e_c
  // (Galerkin: P^T A_f P = A_c), so each pass starts the coarse cycle from zero
  const int passes = (l - 1 == 0) ? 1 : h->prm.cycle;
  for (int g = 0; g < passes; ++g) {
    sv::launch_apply<R>(L.d, cur, b, Buf<R>::r(L), 1, s);
    sv::launch_restrict<R>(L.d, C.d, Buf<R>::r(L), Buf<R>::b(C), s);
    vcycle<R>(h, l - 1, Buf<R>::b(C), Buf<R>::e(C));
    sv::launch_prolong_add<R>(L.d, C.d, Buf<R>::e(C), cur, s);
  }
  for (int it = 0; it < h->prm.nu2; ++it) {
    R* dst = (it == h->prm.nu2 - 1) ? out : ((cur == X0) ? X1 : X0);
    timed_sweep<R>(h, finest, L, cur, b, dst);
    cur = dst;
  }
  if (h->prm.nu2 == 0) cudaMemcpyAsync(out, cur, L.d.N * sizeof(R), cudaMemcpyDeviceToDevice, s);
}

// ---- block-triangular preconditioner (Section 3.4, Algorithm 5) ----
// One V(nu, nu) cycle of scalar multigrid on block blk (0: velocity Laplacian L,
// 1: pressure mass M) with weighted Jacobi, zero initial guess, exact coarse solve.
// Vectors keep the full [u_x | u_y | p] layout with the other block at zero; the
// velocity residual uses the Stokes operator, whose B^T p term then vanishes.
void bt_vcycle(stokes_hierarchy* h, int blk, int l, const double* b, double* out) {
  cudaStream_t s = h->stream;
  sv::Level& L = h->lv[l];
  if (l == 0) {
    cudaMemsetAsync(out, 0, L.d.N * sizeof(double), s);
    if (blk == 0)
      sv::launch_coarse(h->bt_GL, h->bt_nL, b, out, s);
    else
      sv::launch_coarse(h->bt_GM, h->bt_nM, b + 2 * L.d.nv, out + 2 * L.d.nv, s);
    return;
  }
  const double om = (blk == 0) ? h->prm.bt_omega_u : h->prm.bt_omega_p;
  auto resid = [&](const double* x, double* r) {
    if (blk == 0)
      sv::launch_apply<double>(L.d, x, b, r, 1, s);
    else
      sv::launch_mass_resid(L.d, x, b, r, s);
  };
  auto smooth = [&](double*& cur, double* dst) {
    if (cur == nullptr) {
      sv::launch_block_jacobi(L.d, blk, nullptr, b, dst, om, s);
    } else {
      resid(cur, L.r);
      sv::launch_block_jacobi(L.d, blk, cur, L.r, dst, om, s);
    }
    cur = dst;
  };
  double* cur = nullptr;
  for (int it = 0; it < h->prm.bt_nu; ++it) smooth(cur, (cur == L.x0) ? L.x1 : L.x0);
  if (cur == nullptr) {
    cudaMemsetAsync(L.x0, 0, L.d.N * sizeof(double), s);
    cur = L.x0;
  }
  sv::Level& C = h->lv[l - 1];
  resid(cur, L.r);
  sv::launch_restrict<double>(L.d, C.d, L.r, C.b, s);
  bt_vcycle(h, blk, l - 1, C.b, C.e);
  sv::launch_prolong_add<double>(L.d, C.d, C.e, cur, s);
  for (int it = 0; it < h->prm.bt_nu; ++it) smooth(cur, (it == h->prm.bt_nu - 1) ? out : ((cur == L.x0) ? L.x1 : L.x0));
  if (h->prm.bt_nu == 0) cudaMemcpyAsync(out, cur, L.d.N * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

// z = P_BT^-1 r: dp from bt_cycles cycles on M dp = -r_p, then du from bt_cycles
// cycles on L du = r_u - B^T dp (iterative refinement from zero).
void bt_precondition(stokes_hierarchy* h, const double* r, double* z) {
  cudaStream_t s = h->stream;
  const int top = static_cast<int>(h->lv.size()) - 1;
  sv::Level& F = h->lv[top];
  const long long N = F.d.N, nvel = 2 * F.d.nv;
  double* rhs = h->bt_buf;
  double* tmp = rhs + N;
  double* acc = tmp + N;
  // 1. M dp = -r_p (rhs = (0, -r_p)), accumulated in z = (0, dp)
  sv::launch_scale(rhs, r, nullptr, -1.0, N, s);
  cudaMemsetAsync(rhs, 0, nvel * sizeof(double), s);
  cudaMemsetAsync(z, 0, N * sizeof(double), s);
  for (int c = 0; c < h->prm.bt_cycles; ++c) {
    sv::launch_mass_resid(F.d, c == 0 ? nullptr : z, rhs, tmp, s);
    bt_vcycle(h, 1, top, tmp, F.e);
    sv::launch_add(z, F.e, N, s);
  }
  // 2. L du = r_u - B^T dp: rhs = r - A (0, dp) on the velocity rows
  sv::launch_apply<double>(F.d, z, r, rhs, 1, s);
  cudaMemsetAsync(acc, 0, N * sizeof(double), s);
  for (int c = 0; c < h->prm.bt_cycles; ++c) {
    const double* in = rhs;
    if (c > 0) {
      sv::launch_apply<double>(F.d, acc, rhs, tmp, 1, s);
      in = tmp;
    }
    bt_vcycle(h, 0, top, in, F.e);
    sv::launch_add(acc, F.e, N, s);
  }
  cudaMemcpyAsync(z, acc, nvel * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

// z = MG(r) on the finest level in the hierarchy's precision.  The mixed form
// converts r to FP32, cycles in FP32 and converts the result back to FP64.
void precondition(stokes_hierarchy* h, const double* r, double* z) {
  const int top = static_cast<int>(h->lv.size()) - 1;
  ++h->vcycles;
  if (h->prm.precond == 1) {
    bt_precondition(h, r, z);
    return;
  }
  if (h->prm.prec == STOKES_FP64 || top == 0) {
    vcycle<double>(h, top, r, z);
    return;
  }
  sv::Level& F = h->lv[top];
  sv::launch_convert<double, float>(r, F.bf, F.d.N, h->stream);
  vcycle<float>(h, top, F.bf, F.ef);
  sv::launch_convert<float, double>(F.ef, z, F.d.N, h->stream);
}

stokes_status read_scalar(stokes_hierarchy* h, const double* dev, double* out) {
  SV_TRY(cudaMemcpyAsync(h->host_scalars, dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
         "copy scalar");
  SV_TRY(cudaMemcpyAsync(h->host_scalars + 1, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
         "copy error flag");
  SV_TRY(cudaStreamSynchronize(h->stream), "stream sync");
  *out = h->host_scalars[0];
  int flag = 0;
  std::memcpy(&flag, h->host_scalars + 1, sizeof(int));
  if (flag != 0) {
    // reported once: the flag (and the grid-barrier state) is cleared so that the
    // hierarchy stays usable
    cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream);
    if (h->tail_bar) cudaMemsetAsync(h->tail_bar, 0, 2 * sizeof(unsigned), h->stream);
    return fail(STOKES_ERR_TIMEOUT, "a bounded device wait expired (tensor-core sweep or grid barrier)");
  }
  return STOKES_OK;
}

struct SmallBuf {
  double *H, *g, *cs, *sn, *hcol, *h2, *y, *sc;
};

SmallBuf small_layout(stokes_hierarchy* h) {
  const int m = h->m;
  SmallBuf s;
  s.H = h->small;
  s.g = s.H + (m + 1) * m;
  s.cs = s.g + (m + 1);
  s.sn = s.cs + m;
  s.hcol = s.sn + m;
  s.h2 = s.hcol + (m + 1);
  s.y = s.h2 + (m + 1);
  s.sc = s.y + m;
  return s;
}

// H ((m+1) m), g (m+1), cs (m), sn (m), hcol (m+1), h2 (m+1), y (m), 8 scalars
size_t small_size(int m) { return static_cast<size_t>((m + 1) * m + 6 * m + 3 + 8); }


}  // namespace

// ---- FGMRES(m), right-preconditioned (Section 6.8), as stream-ordered pieces ----
// The pieces launch on h->stream and never synchronise, so a batch can run
// them on many streams and capture iterations into CUDA graphs.
namespace sv {

double* fg_scalars(stokes_hierarchy* h) { return small_layout(h).sc; }

// V_0 = b - A x, sc[0] = ||V_0||^2
void fg_residual(stokes_hierarchy* h, const double* b, const double* x) {
  sv::Level& F = h->lv.back();
  const long long N = F.d.N;
  SmallBuf sb = small_layout(h);
  sv::launch_apply<double>(F.d, x, b, h->V, 1, h->stream);
  sv::launch_orth_dots(h->V, N, 0, h->V, N, h->partials, h->npart, h->ticket, nullptr, sb.sc, nullptr,
                       h->stream);
}

// V_0 /= beta, g = beta e_1 (beta known on the host)
void fg_start_cycle(stokes_hierarchy* h, double beta) {
  const long long N = h->lv.back().d.N;
  SmallBuf sb = small_layout(h);
  sv::launch_scale(h->V, h->V, nullptr, 1.0 / beta, N, h->stream);
  sv::launch_fill(sb.g, 0.0, h->m + 1, h->stream);
  sv::launch_fill(sb.g, beta, 1, h->stream);
}

// iteration j: Z_j = MG(V_j), w = A Z_j, Gram-Schmidt against V_0..V_j,
// V_{j+1} = w / ||w||, Givens rotation j; sc[2] = |g_{j+1}| (the residual
// estimate).  Gram-Schmidt is modified (one pass per basis vector) or classical
// (a second pass when the first removed more than half of ||w||^2: the DGKS
// test, taken on the device), by stokes_params.orth.  Scalars: sc[0..1] =
// ||w||^2, ||w||; sc[3..4] = ||A Z_j||^2 and its root; sc[5] = 1 if the
// classical second pass runs.
void fg_iteration(stokes_hierarchy* h, int j) {
  cudaStream_t s = h->stream;
  sv::Level& F = h->lv.back();
  const long long N = F.d.N, ld = N;
  const int m = h->m;
  SmallBuf sb = small_layout(h);
  double* V = h->V;
  double* vj = V + j * ld;
  double* zj = h->Z + j * ld;
  double* w = V + (j + 1) * ld;
  precondition(h, vj, zj);
  sv::launch_apply<double>(F.d, zj, nullptr, w, 0, s);
  double* P = h->partials;
  const int np = h->npart;
  if (h->prm.orth == 2 || (h->prm.orth == 0 && N >= (1LL << 20))) {
    // modified Gram-Schmidt: h_0 = <V_0, w> with ||w||^2 (sc[3..4]); then
    // w -= h_{i-1} V_{i-1} and h_i = <V_i, w> for i = 1..j; last, w -= h_j V_j
    // and the new ||w||^2 (sc[0..1])
    sv::launch_mgs_step(w, nullptr, V, nullptr, N, P, np, h->ticket, sb.hcol, sb.sc + 3, s);
    for (int i = 1; i <= j; ++i)
      sv::launch_mgs_step(w, V + (i - 1) * ld, V + i * ld, sb.hcol + (i - 1), N, P, np, h->ticket, sb.hcol + i,
                          nullptr, s);
    sv::launch_mgs_step(w, V + j * ld, nullptr, sb.hcol + j, N, P, np, h->ticket, nullptr, sb.sc, s);
    sv::launch_scale(w, w, sb.sc + 1, 0.0, N, s);
    sv::launch_givens(sb.H, m + 1, sb.cs, sb.sn, sb.g, sb.hcol, sb.sc + 1, j, sb.sc + 2, s);
    return;
  }
  // classical: pass 1: h = V^T w and ||w||^2; w -= V h with the new ||w||^2 and the DGKS
  // flag, fused (up to 16 basis vectors) with pass 2's dots h2 = V^T w
  sv::launch_orth_dots(V, ld, j + 1, w, N, P, np, h->ticket, sb.hcol, sb.sc + 3, nullptr, s);
  if (!sv::launch_orth_update_dots(w, V, ld, j + 1, sb.hcol, N, P, np, h->ticket, sb.h2, sb.sc, sb.sc + 3,
                                   sb.sc + 5, s)) {
    sv::launch_orth_update(w, V, ld, j + 1, sb.hcol, N, P, np, h->ticket, sb.sc, nullptr, sb.sc + 3,
                           sb.sc + 5, nullptr, s);
    sv::launch_orth_dots(V, ld, j + 1, w, N, P, np, h->ticket, sb.h2, nullptr, sb.sc + 5, s);
  }
  // pass 2, only where flagged: w -= V h2, h += h2
  sv::launch_orth_update(w, V, ld, j + 1, sb.h2, N, P, np, h->ticket, sb.sc, sb.sc + 5, nullptr, nullptr,
                         sb.hcol, s);
  sv::launch_scale(w, w, sb.sc + 1, 0.0, N, s);
  sv::launch_givens(sb.H, m + 1, sb.cs, sb.sn, sb.g, sb.hcol, sb.sc + 1, j, sb.sc + 2, s);
}

// end of a cycle after k iterations: y = H_k^-1 g, x += Z y, then fg_residual
void fg_finish_cycle(stokes_hierarchy* h, int k, const double* b, double* x) {
  const long long N = h->lv.back().d.N;
  SmallBuf sb = small_layout(h);
  sv::launch_backsolve(sb.H, h->m + 1, sb.g, k, sb.y, h->stream);
  sv::launch_multiaxpy(x, h->Z, N, k, sb.y, 1.0, N, h->stream);
  fg_residual(h, b, x);
}

}  // namespace sv

namespace {

stokes_status fgmres(stokes_hierarchy* h, const double* b, double* x, int* iters_out,
                     double* relres_out) {
  double* sc = sv::fg_scalars(h);
  int it = 0;
  double beta0 = 0.0, beta = 0.0, v2 = 0.0;
  stokes_status st;
  sv::fg_residual(h, b, x);
  if ((st = check_launch("fgmres residual")) != STOKES_OK) return st;
  if ((st = read_scalar(h, sc, &v2)) != STOKES_OK) return st;
  beta0 = std::sqrt(v2);
  if (!std::isfinite(beta0)) return fail(STOKES_ERR_NONFINITE, "initial residual is not finite");
  if (iters_out) *iters_out = 0;
  if (relres_out) *relres_out = 0.0;
  if (beta0 == 0.0) return STOKES_OK;
  beta = beta0;
  const double tol = h->prm.rtol * beta0;
  stokes_status result = STOKES_NOT_CONVERGED;
  while (true) {
    sv::fg_start_cycle(h, beta);
    int k = 0;
    for (int j = 0; j < h->m; ++j) {
      sv::fg_iteration(h, j);
      if ((st = check_launch("fgmres iteration")) != STOKES_OK) return st;
      double est;
      if ((st = read_scalar(h, sc + 2, &est)) != STOKES_OK) return st;
      ++it;
      k = j + 1;
      if (!std::isfinite(est)) return fail(STOKES_ERR_NONFINITE, "residual estimate is not finite");
      if (est <= tol || it >= h->prm.maxit) break;
    }
    sv::fg_finish_cycle(h, k, b, x);
    if ((st = check_launch("fgmres update")) != STOKES_OK) return st;
    if ((st = read_scalar(h, sc, &v2)) != STOKES_OK) return st;
    beta = std::sqrt(v2);
    if (!std::isfinite(beta)) return fail(STOKES_ERR_NONFINITE, "residual is not finite");
    if (beta <= tol) {
      result = STOKES_OK;
      break;
    }
    if (it >= h->prm.maxit) break;
  }
  if (iters_out) *iters_out = it;
  if (relres_out) *relres_out = beta / beta0;
  if (result == STOKES_NOT_CONVERGED) return fail(result, "FGMRES reached maxit");
  return STOKES_OK;
}

// Tile shape of the sweep per level and precision: fixed by params.tile, or
// (tile = -1) the fastest of the shapes on that level, timed with CUDA events
// on the hierarchy's stream.  Every level with sweeps is tuned: on the small
// ones the 4 x 4 tile spreads the FP64 patch solves over more SMs.
template <typename R>
cudaError_t tune_level(stokes_hierarchy* h, sv::Level& L, int* cfg) {
  cudaStream_t s = h->stream;
  R* x = Buf<R>::x0(L);
  R* b = Buf<R>::b(L);
  R* xo = Buf<R>::x1(L);
  const R* cd = nullptr;
  cudaError_t e;
  if ((e = cudaMemsetAsync(x, 0, L.d.N * sizeof(R), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b, 0, L.d.N * sizeof(R), s)) != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  float best = 1e30f;
  // candidates: the fused tile shapes; in FP64 also the split sweep; in the mixed
  // forms, on levels with interior strips, also the strip sweep with its ring
  const bool tc = (sizeof(R) == 4) && L.strip;
  constexpr int CAND_TC = sv::VANKA_CFG_4 + 1;   // the strip sweep (mixed forms), tuning index only
  const int ncand = tc ? CAND_TC + 1 : sv::VANKA_CFG_4 + 1;
  int best_c = 0;
  for (int c = 0; c < ncand; ++c) {
    if (tc && c == sv::VANKA_CFG_14) continue;   // where the strip tiles fit, 14x14 means the strip sweep
    auto run = [&]() {
      if constexpr (sizeof(R) == 8) {
        if (sv::vanka_cfg_split(c))
          sv::launch_vanka_split<double>(L.d, L.cd, h->fd, x, b, xo, h->prm.omega, h->delta,
                                         c == sv::VANKA_CFG_SPLIT2, s, L.r);
        else
          sv::launch_vanka<double>(L.d, L.cd, h->fd, x, b, xo, h->prm.omega, c, s);
      } else {
        if (c == CAND_TC) {
          tc_sweep(h, L, x, b, xo, s);
        } else if (sv::vanka_cfg_split(c)) {
          sv::launch_vanka_split<float>(L.d, L.cdf, h->fdf, x, b, xo, h->prm.omega, h->deltaf,
                                        c == sv::VANKA_CFG_SPLIT2, s, nullptr);
        } else {
          sv::launch_vanka<float>(L.d, L.cdf, h->fdf, x, b, xo, h->prm.omega, c, s);
        }
      }
    };
    // one untimed run, then the best of three timed trials: a trial is a few sweeps
    // on large levels and more on small ones, where one sweep lasts microseconds and
    // a single trial is at the mercy of launch jitter
    run();
    const int reps = L.d.N > (1 << 22) ? 3 : 10;
    float ms = 1e30f;
    for (int trial = 0; trial < 3 && e == cudaSuccess; ++trial) {
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps; ++r) run();
      cudaEventRecord(e1, s);
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float t = 0.0f;
      cudaEventElapsedTime(&t, e0, e1);
      ms = std::min(ms, t / reps);
    }
    if (e != cudaSuccess) break;
    if (ms < best) {
      best = ms;
      best_c = c;
    }
  }
  if (tc) {   // the strip sweep, or the fastest SIMT configuration
    L.tc_on = (best_c == CAND_TC);
    *cfg = L.tc_on ? sv::VANKA_CFG_14 : best_c;
  } else {
    *cfg = best_c;
  }
  (void)cd;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t choose_tiles(stokes_hierarchy* h) {
  for (sv::Level& L : h->lv) {
    if (h->prm.tile >= 0 || h->prm.smoother != STOKES_SMOOTHER_SHARED || h->prm.precond == 1) {
      L.vk_cfg = L.vk_cfg_f = h->prm.tile >= 0 ? h->prm.tile : 1;   // no tiled sweep runs with per-patch inverses
      L.tc_on = (h->prm.tile == sv::VANKA_CFG_14 || h->prm.tile < 0);
      continue;
    }
    L.vk_cfg = L.vk_cfg_f = (L.d.n < 64) ? 0 : 1;
    if (&L == &h->lv.front()) continue;   // the coarsest level is solved exactly: no sweeps
    if (static_cast<int>(&L - &h->lv.front()) <= h->tail_top) continue;   // swept by the persistent launch
    // only the precision the V-cycle runs in is tuned (the FP64 sweep of a
    // mixed hierarchy serves stokes_vanka_sweep alone and keeps 16x8)
    cudaError_t e = cudaSuccess;
    if (h->prm.prec == STOKES_FP64) e = tune_level<double>(h, L, &L.vk_cfg);
    else e = tune_level<float>(h, L, &L.vk_cfg_f);   // strip sweep vs SIMT shapes
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

namespace sv {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace sv

extern "C" {

void stokes_default_params(stokes_params* p) {
  if (!p) return;
  p->nu1 = 2;
  p->nu2 = 2;
  p->omega = 0.7;
  p->coarse_n = 4;
  p->restart = 30;
  p->maxit = 1000;
  p->rtol = 1e-8;
  p->prec = STOKES_FP64;
  p->tile = -1;
  p->smoother = STOKES_SMOOTHER_SHARED;
  p->bs_t = 1.0;
  p->bs_omega = 1.0;
  p->bs_jacobi_weight = 1.0;
  p->bs_jacobi_iters = 2;
  p->cycle = 1;
  p->precond = 0;
  p->bt_cycles = 3;
  p->bt_nu = 3;
  p->bt_omega_u = 1.0;
  p->bt_omega_p = 0.6;
  p->tail_n = 0;
  p->orth = 0;
}

const char* stokes_last_error(void) { return g_err.c_str(); }

stokes_status stokes_hierarchy_create(int n, double viscosity, const stokes_params* params,
                                      void* stream, stokes_hierarchy** out) {
  g_err.clear();
  if (out == nullptr) return fail(STOKES_ERR_ARG, "out is null");
  *out = nullptr;
  stokes_params prm;
  stokes_default_params(&prm);
  if (params) prm = *params;
  if (!(viscosity > 0.0) || !std::isfinite(viscosity)) return fail(STOKES_ERR_ARG, "viscosity must be > 0");
  if (prm.coarse_n < 4) return fail(STOKES_ERR_ARG, "coarse_n must be >= 4");
  if (prm.restart < 1 || prm.restart > 64) return fail(STOKES_ERR_ARG, "restart must be in 1..64");
  if (prm.nu1 < 0 || prm.nu2 < 0 || prm.maxit < 1 || !(prm.rtol >= 0.0) || !(prm.omega > 0.0))
    return fail(STOKES_ERR_ARG, "bad smoothing / iteration parameters");
  if (prm.prec != STOKES_FP64 && prm.prec != STOKES_MIXED_FP32 && prm.prec != STOKES_MIXED_BF16)
    return fail(STOKES_ERR_ARG, "unknown precision mode");
  if (prm.tile < -1 || prm.tile > sv::VANKA_CFG_4) return fail(STOKES_ERR_ARG, "tile must be -1..6");

  if (prm.cycle < 1 || prm.cycle > 2) return fail(STOKES_ERR_ARG, "cycle must be 1 (V) or 2 (W)");
  if (prm.orth < 0 || prm.orth > 2) return fail(STOKES_ERR_ARG, "orth must be 0 (by size), 1 or 2");
  if (prm.precond < 0 || prm.precond > 1) return fail(STOKES_ERR_ARG, "precond must be 0 or 1");
  if (prm.precond == 1 && (prm.prec != STOKES_FP64 || prm.bt_cycles < 1 || prm.bt_nu < 0 ||
                           !(prm.bt_omega_u > 0.0) || !(prm.bt_omega_p > 0.0)))
    return fail(STOKES_ERR_ARG, "block-triangular preconditioner: FP64, bt_cycles >= 1, bt_nu >= 0, weights > 0");
  if (prm.smoother < STOKES_SMOOTHER_SHARED || prm.smoother > STOKES_SMOOTHER_SCHUR_UZAWA)
    return fail(STOKES_ERR_ARG, "unknown smoother");
  if ((prm.smoother == STOKES_SMOOTHER_BRAESS_SARAZIN || prm.smoother == STOKES_SMOOTHER_SCHUR_UZAWA) &&
      (prm.prec == STOKES_MIXED_BF16 || !(prm.bs_t > 0.0) || !(prm.bs_omega > 0.0) ||
       !(prm.bs_jacobi_weight > 0.0) || prm.bs_jacobi_iters < 1 || prm.bs_jacobi_iters > 64))
    return fail(STOKES_ERR_ARG, "Braess-Sarazin / Schur-Uzawa: FP64 or mixed FP32, t, omega, weight > 0, 1..64 Jacobi steps");
  if (prm.smoother == STOKES_SMOOTHER_PER_PATCH && prm.prec != STOKES_FP64)
    return fail(STOKES_ERR_ARG, "per-patch inverses (simple Vanka) are FP64 only");
  std::vector<int> sizes;
  {
    int m = n;
    while (m > prm.coarse_n) {
      if (m % 2) return fail(STOKES_ERR_ARG, "n must be coarse_n * 2^k");
      sizes.push_back(m);
      m /= 2;
    }
    if (m != prm.coarse_n) return fail(STOKES_ERR_ARG, "n must be coarse_n * 2^k");
    sizes.push_back(m);
  }
  auto* h = new (std::nothrow) stokes_hierarchy();
  if (!h) return fail(STOKES_ERR_OOM, "host allocation failed");
  t_alloc_used = 0;
  h->prm = prm;
  h->bs.t = prm.bs_t;
  h->bs.omega = prm.bs_omega;
  h->bs.jacobi_weight = prm.bs_jacobi_weight;
  h->bs.jacobi_iters = prm.bs_jacobi_iters;
  h->bs.uzawa = (prm.smoother == STOKES_SMOOTHER_SCHUR_UZAWA);
  h->nu = viscosity;
  h->n = n;
  h->stream = static_cast<cudaStream_t>(stream);
  h->m = prm.restart;
  h->fd = sv::interior_fast_diag(viscosity);
  h->fdf = sv::fd_cast<float>(h->fd, [](double v) { return static_cast<float>(v); });
  cudaError_t e = sv::vanka_prepare();
  if (e == cudaSuccess) e = sv::simple_prepare();
  if (e == cudaSuccess) {
    static std::once_flag z_once;
    static cudaError_t z_err = cudaSuccess;
    std::call_once(z_once, [] {
      z_err = sv::set_interior_unit_z(unit_schur().z);
      if (z_err == cudaSuccess) z_err = sv::set_strip_unit_z(unit_schur().z);
    });
    e = z_err;
  }
  const bool mixed = prm.prec == STOKES_MIXED_BF16 || prm.prec == STOKES_MIXED_FP32;
  if (e == cudaSuccess && mixed) e = sv::vanka_tc_prepare();
  if (e == cudaSuccess && mixed) {
    e = cudaStreamCreateWithFlags(&h->ring_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ring_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ring_join, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    free_all(h);
    delete h;
    return cuda_fail(e, "kernel attributes");
  }
  h->lv.resize(sizes.size());
  for (size_t k = 0; k < sizes.size(); ++k) {
    sv::Level& L = h->lv[k];
    const int nl = sizes[sizes.size() - 1 - k];
    L.d = make_level(nl, viscosity);
    const size_t N = static_cast<size_t>(L.d.N);
    // FP64 level vectors serve the FP64 V-cycle and, on level 0, the exact coarse
    // solve of every form; a mixed-precision hierarchy needs them nowhere else
    const bool f64 = (prm.prec == STOKES_FP64) || k == 0;
    if ((f64 && ((e = dalloc(&L.x0, N)) != cudaSuccess || (e = dalloc(&L.x1, N)) != cudaSuccess ||
                 (e = dalloc(&L.b, N)) != cudaSuccess || (e = dalloc(&L.r, N)) != cudaSuccess ||
                 (e = dalloc(&L.e, N)) != cudaSuccess)) ||
        (e = dalloc(&L.cd, static_cast<size_t>(sv::CD_TOTAL))) != cudaSuccess) {
      free_all(h);
      delete h;
      return cuda_fail(e, "level allocation");
    }
    sv::build_class_data(nl, viscosity, L.cd_host, &L.full_inv_host);
    e = cudaMemcpy(L.cd, L.cd_host.data(), L.cd_host.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && mixed) {
      sv::tc_interior_range(nl, &L.tc_lo, &L.tc_hi);
      L.strip = L.tc_hi >= L.tc_lo;
      if (L.strip && prm.prec == STOKES_MIXED_BF16) {
        std::vector<unsigned short> img(64 * 64);
        sv::tc_pack_inverse(L.full_inv_host.data() + static_cast<size_t>(sv::INTERIOR_CLASS) * 51 * 51, img.data());
        if ((e = dalloc_bytes(&L.tcB, img.size() * sizeof(unsigned short))) == cudaSuccess)
          e = cudaMemcpy(L.tcB, img.data(), img.size() * sizeof(unsigned short), cudaMemcpyHostToDevice);
      }
    }
    if (e == cudaSuccess && prm.smoother == STOKES_SMOOTHER_PER_PATCH) {
      // simple Vanka: assemble and invert every patch of this level on the device
      if ((e = dalloc(&L.pinv, sv::patch_inverse_doubles(L.d))) == cudaSuccess) {
        sv::launch_patch_inverse(L.d, L.pinv, h->stream);
        e = cudaGetLastError();
      }
    }
    // patch corrections of the per-patch-inverse and the split sweeps (finest-level size)
    if (e == cudaSuccess && prm.prec == STOKES_FP64 && k + 1 == sizes.size())
      e = dalloc(&h->delta, std::max(sv::patch_delta_doubles(L.d), sv::split_delta_doubles(L.d)));
    if (e == cudaSuccess && prm.prec != STOKES_FP64 && k + 1 == sizes.size())
      e = dalloc(&h->deltaf, std::max(sv::patch_delta_doubles(L.d), sv::split_delta_doubles(L.d)));
    if (e == cudaSuccess && (prm.smoother == STOKES_SMOOTHER_BRAESS_SARAZIN ||
                             prm.smoother == STOKES_SMOOTHER_SCHUR_UZAWA) && k + 1 == sizes.size()) {
      const size_t el = sv::bs_scratch_elems(L.d) * (prm.prec == STOKES_FP64 ? sizeof(double) : sizeof(float));
      e = dalloc_bytes(&h->bs_buf, el);
    }
    if (e == cudaSuccess && prm.prec != STOKES_FP64) {
      std::vector<float> cdf(L.cd_host.begin(), L.cd_host.end());
      if ((e = dalloc(&L.xf0, N)) == cudaSuccess && (e = dalloc(&L.xf1, N)) == cudaSuccess &&
          (e = dalloc(&L.bf, N)) == cudaSuccess && (e = dalloc(&L.rf, N)) == cudaSuccess &&
          (e = dalloc(&L.ef, N)) == cudaSuccess && (e = dalloc(&L.cdf, cdf.size())) == cudaSuccess)
        e = cudaMemcpy(L.cdf, cdf.data(), cdf.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
      free_all(h);
      delete h;
      return cuda_fail(e, "level data allocation / upload");
    }
  }
  {
    std::vector<double> G;
    if (!sv::coarse_inverse(prm.coarse_n, viscosity, G)) {
      free_all(h);
      delete h;
      return fail(STOKES_ERR_ARG, "coarse bordered system is singular");
    }
    h->N0 = static_cast<int>(h->lv[0].d.N);
    if ((e = dalloc(&h->coarse_G, G.size())) != cudaSuccess ||
        (e = cudaMemcpy(h->coarse_G, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice)) !=
            cudaSuccess) {
      free_all(h);
      delete h;
      return cuda_fail(e, "coarse inverse upload");
    }
  }
  if (prm.precond == 1) {
    std::vector<double> GL, GM;
    if (!sv::bt_coarse_inverses(prm.coarse_n, viscosity, GL, GM)) {
      free_all(h);
      delete h;
      return fail(STOKES_ERR_ARG, "coarse Laplacian or mass matrix is singular");
    }
    h->bt_nL = static_cast<int>(2 * h->lv[0].d.nv);
    h->bt_nM = h->lv[0].d.np * h->lv[0].d.np;
    const size_t Nf = static_cast<size_t>(h->lv.back().d.N);
    if ((e = dalloc(&h->bt_GL, GL.size())) != cudaSuccess || (e = dalloc(&h->bt_GM, GM.size())) != cudaSuccess ||
        (e = dalloc(&h->bt_buf, 3 * Nf)) != cudaSuccess ||
        (e = cudaMemcpy(h->bt_GL, GL.data(), GL.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->bt_GM, GM.data(), GM.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) {
      free_all(h);
      delete h;
      return cuda_fail(e, "block-triangular set-up");
    }
  }
  const size_t Nf = static_cast<size_t>(h->lv.back().d.N);
  h->npart = sv::dot_blocks();
  if ((e = dalloc(&h->V, Nf * (h->m + 1))) != cudaSuccess || (e = dalloc(&h->Z, Nf * h->m)) != cudaSuccess ||
      (e = dalloc(&h->small, small_size(h->m))) != cudaSuccess ||
      (e = dalloc(&h->partials, static_cast<size_t>(h->npart) * 64)) != cudaSuccess ||
      (e = dalloc(&h->dev_err, 1)) != cudaSuccess || (e = dalloc(&h->aux, Nf)) != cudaSuccess ||
      (e = cudaMemset(h->dev_err, 0, sizeof(int))) != cudaSuccess ||
      (e = dalloc(&h->ticket, 1)) != cudaSuccess || (e = cudaMemset(h->ticket, 0, sizeof(unsigned))) != cudaSuccess ||
      (e = cudaMallocHost(reinterpret_cast<void**>(&h->host_scalars), 8 * sizeof(double))) != cudaSuccess) {
    free_all(h);
    delete h;
    return cuda_fail(e, "Krylov workspace allocation");
  }
  if ((e = tail_setup(h)) != cudaSuccess) {
    free_all(h);
    delete h;
    return cuda_fail(e, "persistent coarse-level set-up");
  }
  if ((e = choose_tiles(h)) != cudaSuccess) {
    free_all(h);
    delete h;
    return cuda_fail(e, "tile autotuning");
  }
  *out = h;
  return STOKES_OK;
}

stokes_status stokes_level_tile(const stokes_hierarchy* h, int level, int* tile) {
  stokes_status st = check_level(h, level);
  if (st != STOKES_OK) return st;
  if (tile) *tile = (h->prm.prec == STOKES_FP64) ? h->lv[level].vk_cfg : h->lv[level].vk_cfg_f;
  return STOKES_OK;
}

stokes_status stokes_stats_enable_timing(stokes_hierarchy* h, int enable) {
  if (!h) return fail(STOKES_ERR_ARG, "null hierarchy");
  h->timing = enable != 0;
  return STOKES_OK;
}

stokes_status stokes_stats_reset(stokes_hierarchy* h) {
  if (!h) return fail(STOKES_ERR_ARG, "null hierarchy");
  SV_TRY(cudaStreamSynchronize(h->stream), "stats reset");
  h->ev_used = 0;
  h->sweeps_timed = 0;
  h->sweep_ms = 0.0;
  h->vcycles = 0;
  return STOKES_OK;
}

stokes_status stokes_stats_read(stokes_hierarchy* h, stokes_stats* out) {
  if (!h || !out) return fail(STOKES_ERR_ARG, "null argument");
  SV_TRY(cudaStreamSynchronize(h->stream), "stats read");
  for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
    float ms = 0.0f;
    SV_TRY(cudaEventElapsedTime(&ms, h->ev_pool[k], h->ev_pool[k + 1]), "event elapsed");
    h->sweep_ms += ms;
    ++h->sweeps_timed;
  }
  h->ev_used = 0;
  out->kernel_launches = sv::g_launches.load();
  out->tc_launches = sv::g_tc_launches.load();
  out->vcycles = h->vcycles;
  out->sweeps_timed = h->sweeps_timed;
  out->sweep_ms = h->sweep_ms;
  return STOKES_OK;
}

stokes_status stokes_hierarchy_destroy(stokes_hierarchy* h) {
  if (!h) return STOKES_OK;
  cudaStreamSynchronize(h->stream);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear();
  free_all(h);
  delete h;
  return STOKES_OK;
}

stokes_status stokes_level_info(const stokes_hierarchy* h, int* num_levels, int* n_finest) {
  if (!h) return fail(STOKES_ERR_ARG, "null hierarchy");
  if (num_levels) *num_levels = static_cast<int>(h->lv.size());
  if (n_finest) *n_finest = h->n;
  return STOKES_OK;
}

stokes_status stokes_level_n(const stokes_hierarchy* h, int level, int* n_level) {
  stokes_status st = check_level(h, level);
  if (st != STOKES_OK) return st;
  if (n_level) *n_level = h->lv[level].d.n;
  return STOKES_OK;
}

stokes_status stokes_assemble_rhs(stokes_hierarchy* h, const double* f_nodal, const double* u_dirichlet,
                                  double* b) {
  if (!h || !f_nodal || !u_dirichlet || !b) return fail(STOKES_ERR_ARG, "null argument");
  sv::launch_rhs(h->lv.back().d, f_nodal, u_dirichlet, b, h->stream);
  return check_launch("assemble_rhs");
}

stokes_status stokes_rhs_transpose(stokes_hierarchy* h, const double* lambda, double* grad_f) {
  if (!h || !lambda || !grad_f) return fail(STOKES_ERR_ARG, "null argument");
  sv::launch_rhs_transpose(h->lv.back().d, lambda, grad_f, h->stream);
  return check_launch("rhs_transpose");
}

stokes_status stokes_apply_operator(stokes_hierarchy* h, int level, const double* x, double* y) {
  stokes_status st = check_level(h, level);
  if (st != STOKES_OK) return st;
  if (!x || !y) return fail(STOKES_ERR_ARG, "null vector");
  sv::launch_apply<double>(h->lv[level].d, x, nullptr, y, 0, h->stream);
  return check_launch("apply_operator");
}

stokes_status stokes_residual(stokes_hierarchy* h, int level, const double* b, const double* x, double* r) {
  stokes_status st = check_level(h, level);
  if (st != STOKES_OK) return st;
  if (!x || !b || !r) return fail(STOKES_ERR_ARG, "null vector");
  sv::launch_apply<double>(h->lv[level].d, x, b, r, 1, h->stream);
  return check_launch("residual");
}

stokes_status stokes_vanka_sweep(stokes_hierarchy* h, int level, const double* x, const double* b,
                                 double* x_out) {
  stokes_status st = check_level(h, level);
  if (st != STOKES_OK) return st;
  if (!b || !x_out) return fail(STOKES_ERR_ARG, "null vector");
  if (x_out == x || x_out == b) return fail(STOKES_ERR_ARG, "x_out must not alias x or b");
  sv::Level& L = h->lv[level];
  sweep_f64(h, L, x, b, x_out);
  return check_launch("vanka_sweep");
}

stokes_status stokes_relaxation_sweep(stokes_hierarchy* h, int level, const double* x, const double* b,
                                      double* x_out) {
  stokes_status st = check_level(h, level);
  if (st != STOKES_OK) return st;
  if (!b || !x_out) return fail(STOKES_ERR_ARG, "null vector");
  if (x_out == x || x_out == b) return fail(STOKES_ERR_ARG, "x_out must not alias x or b");
  sv::Level& L = h->lv[level];
  if (h->prm.prec == STOKES_FP64) {
    sweep_f64(h, L, x, b, x_out);
    return check_launch("relaxation_sweep");
  }
  // the mixed forms: round x and b to FP32, sweep in the V-cycle's arithmetic, widen the result
  const long long N = L.d.N;
  sv::launch_convert<double, float>(b, L.bf, N, h->stream);
  if (x) sv::launch_convert<double, float>(x, L.xf0, N, h->stream);
  timed_sweep<float>(h, false, L, x ? L.xf0 : nullptr, L.bf, L.xf1);
  sv::launch_convert<float, double>(L.xf1, x_out, N, h->stream);
  return check_launch("relaxation_sweep");
}

stokes_status stokes_device_status(stokes_hierarchy* h) {
  if (!h) return fail(STOKES_ERR_ARG, "null hierarchy");
  SV_TRY(cudaMemcpyAsync(h->host_scalars + 1, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
         "copy error flag");
  SV_TRY(cudaStreamSynchronize(h->stream), "stream sync");
  int flag = 0;
  std::memcpy(&flag, h->host_scalars + 1, sizeof(int));
  if (flag != 0) {
    SV_TRY(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream), "clear error flag");
    if (h->tail_bar) SV_TRY(cudaMemsetAsync(h->tail_bar, 0, 2 * sizeof(unsigned), h->stream), "reset grid barrier");
    return fail(STOKES_ERR_TIMEOUT, "a bounded device wait expired (tensor-core sweep or grid barrier)");
  }
  return STOKES_OK;
}

stokes_status stokes_test_set_wait_limit(stokes_hierarchy* h, int polls) {
  if (!h) return fail(STOKES_ERR_ARG, "null hierarchy");
  h->tc_wait_limit = (polls < 0 || polls > sv::TC_WAIT_LIMIT) ? sv::TC_WAIT_LIMIT : polls;
  return STOKES_OK;
}

void stokes_test_set_alloc_limit(long long bytes) { g_alloc_cap.store(bytes > 0 ? bytes : 0); }

stokes_status stokes_test_set_grid_barrier(stokes_hierarchy* h, int polls, int withhold_cta) {
  if (!h) return fail(STOKES_ERR_ARG, "null hierarchy");
  h->tail_spin_limit = (polls < 0 || polls > sv::TAIL_SPIN_LIMIT) ? sv::TAIL_SPIN_LIMIT : polls;
  h->tail_skip_arrival = withhold_cta >= 0 ? withhold_cta : -1;
  return STOKES_OK;
}

stokes_status stokes_tail_info(const stokes_hierarchy* h, int* top_level, int* steps, int* ctas) {
  if (!h) return fail(STOKES_ERR_ARG, "null hierarchy");
  if (top_level) *top_level = h->tail_top;
  if (steps) *steps = h->tail_nops;
  if (ctas) *ctas = h->tail_grid;
  return STOKES_OK;
}

stokes_status stokes_restrict(stokes_hierarchy* h, int level, const double* r_fine, double* r_coarse) {
  stokes_status st = check_level(h, level, 1);
  if (st != STOKES_OK) return st;
  if (!r_fine || !r_coarse) return fail(STOKES_ERR_ARG, "null vector");
  sv::launch_restrict<double>(h->lv[level].d, h->lv[level - 1].d, r_fine, r_coarse, h->stream);
  return check_launch("restrict");
}

stokes_status stokes_prolong_add(stokes_hierarchy* h, int level, const double* e_coarse, double* x_fine) {
  stokes_status st = check_level(h, level, 1);
  if (st != STOKES_OK) return st;
  if (!e_coarse || !x_fine) return fail(STOKES_ERR_ARG, "null vector");
  sv::launch_prolong_add<double>(h->lv[level].d, h->lv[level - 1].d, e_coarse, x_fine, h->stream);
  return check_launch("prolong_add");
}

stokes_status stokes_coarse_solve(stokes_hierarchy* h, const double* r, double* e) {
  if (!h || !r || !e) return fail(STOKES_ERR_ARG, "null argument");
  if (r == e) return fail(STOKES_ERR_ARG, "r and e must not alias");
  sv::launch_coarse(h->coarse_G, h->N0, r, e, h->stream);
  return check_launch("coarse_solve");
}

stokes_status stokes_initial_guess(stokes_hierarchy* h, const double* b, double* x0) {
  if (!h || !b || !x0) return fail(STOKES_ERR_ARG, "null argument");
  if (b == x0) return fail(STOKES_ERR_ARG, "b and x0 must not alias");
  sv::launch_dirichlet_copy(h->lv.back().d, b, x0, h->stream);
  return check_launch("initial_guess");
}

stokes_status stokes_vcycle_apply(stokes_hierarchy* h, const double* r, double* z) {
  if (!h || !r || !z) return fail(STOKES_ERR_ARG, "null argument");
  if (r == z) return fail(STOKES_ERR_ARG, "r and z must not alias");
  precondition(h, r, z);
  return check_launch("vcycle");
}

stokes_status stokes_fgmres_solve(stokes_hierarchy* h, const double* b, double* x, int* iters,
                                  double* relres) {
  if (!h || !b || !x) return fail(STOKES_ERR_ARG, "null argument");
  g_err.clear();
  return fgmres(h, b, x, iters, relres);
}

stokes_status stokes_solve_adjoint(stokes_hierarchy* h, const double* g, double* lambda, double* grad_f,
                                   int* iters, double* relres) {
  if (!h || !g || !lambda) return fail(STOKES_ERR_ARG, "null argument");
  if (g == lambda) return fail(STOKES_ERR_ARG, "g and lambda must not alias");
  g_err.clear();
  sv::Level& F = h->lv.back();
  // A^T = A is singular with kernel (0, 1_p): remove the component of g along it
  double* sc = h->small + (h->m + 1) * h->m + 6 * h->m + 3;
  sv::launch_project_pressure(F.d, g, h->aux, h->partials, h->npart, sc, h->stream);
  // initial guess: zero on free rows, g on Dirichlet rows (A has identity rows there)
  sv::launch_dirichlet_copy(F.d, h->aux, lambda, h->stream);
  stokes_status st = fgmres(h, h->aux, lambda, iters, relres);
  if (st != STOKES_OK) return st;
  if (grad_f) {
    sv::launch_rhs_transpose(F.d, lambda, grad_f, h->stream);
    return check_launch("rhs_transpose");
  }
  return STOKES_OK;
}

stokes_status stokes_batched_solve(stokes_hierarchy* const* hs, int nprob, const double* const* b,
                                   double* const* x, int* iters, double* relres) {
  if (!hs || nprob < 0 || (nprob > 0 && (!b || !x))) return fail(STOKES_ERR_ARG, "null argument");
  stokes_status first = STOKES_OK;
  for (int k = 0; k < nprob; ++k) {
    stokes_status st = stokes_fgmres_solve(hs[k], b[k], x[k], iters ? iters + k : nullptr,
                                           relres ? relres + k : nullptr);
    if (st != STOKES_OK && first == STOKES_OK) first = st;
  }
  return first;
}

}  // extern "C"
