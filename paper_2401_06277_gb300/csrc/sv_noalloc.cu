// sv_noalloc.cu -- stokes_residual_norm_noalloc: ||b - A x||_2 for callers
// that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden --
// for example a host framework whose device memory is entirely owned by its
// own pool allocator, or a monitoring hook that runs while another component
// is recording work into a stream.  The regular path (stokes_residual into a
// caller buffer, then a norm through the hierarchy's dot-product workspace)
// needs memory that a hierarchy allocated; this entry point needs none.
//
// Its scratch is one file-scope device array (one partial sum per grid row),
// so it supports n <= STOKES_NOALLOC_MAX_N.  Every GPU that loads this
// library holds the array (196.6 KB) until the process exits.  Each call
// overwrites every slot it reads, so nothing has to be cleared between calls;
// calls whose kernels overlap on the GPU (different streams, or different
// host threads) share the array and race.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <mutex>
#include <string>

#include "sv_internal.h"
#include "sv_stencil.cuh"

namespace {

constexpr int NOALLOC_SLOTS = (2 * STOKES_NOALLOC_MAX_N + 1) + (STOKES_NOALLOC_MAX_N + 1);
__device__ __align__(256) double g_noalloc_scratch[NOALLOC_SLOTS];

constexpr int MAX_DEVICES = 64;
// per device: the scratch address and the ID of the context it was looked up in
struct ScratchEntry {
  unsigned long long ctx_id;
  double* addr;
};
ScratchEntry g_scratch[MAX_DEVICES];
std::mutex g_scratch_mutex;

__device__ __forceinline__ bool na_free(int I, int J, int nq) {
  return I > 0 && J > 0 && I < nq - 1 && J < nq - 1;
}

__device__ __forceinline__ double na_block_sum(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// Block r < nq: squared residual of Q2 row J = r (both velocity components);
// block r >= nq: squared residual of vertex row j = r - nq.  Partial -> scratch[r].
__global__ void k_resnorm_rows(sv::LevelDev L, const double* __restrict__ b,
                               const double* __restrict__ x, double* __restrict__ scratch) {
  sv::pdl_begin();
  const int r = blockIdx.x;
  const int nq = L.nq, np = L.np, n = L.n;
  const long long nv = L.nv;
  const double cl = L.nu / 90.0, cb = -L.h / 18.0;
  double acc = 0.0;
  if (r < nq) {
    const int J = r;
    for (int I = threadIdx.x; I < nq; I += blockDim.x) {
      const long long k = static_cast<long long>(J) * nq + I;
      double ax, ay;
      if (!na_free(I, J, nq)) {
        ax = x[k];
        ay = x[nv + k];
      } else {
        double sx = 0.0, sy = 0.0;
        for (int dJ = -2; dJ <= 2; ++dJ) {
          const int J2 = J + dJ;
          if (J2 <= 0 || J2 >= nq - 1) continue;
          const double mJ = sv::m1(J, dJ), kJ = sv::k1(J, dJ);
          for (int dI = -2; dI <= 2; ++dI) {
            const int I2 = I + dI;
            if (I2 <= 0 || I2 >= nq - 1) continue;
            const double c = sv::k1(I, dI) * mJ + sv::m1(I, dI) * kJ;
            const long long kk = static_cast<long long>(J2) * nq + I2;
            sx = fma(c, x[kk], sx);
            sy = fma(c, x[nv + kk], sy);
          }
        }
        double gx = 0.0, gy = 0.0;
        for (int j = J / 2 - 1; j <= J / 2 + 1; ++j) {
          if (j < 0 || j > n) continue;
          for (int i = I / 2 - 1; i <= I / 2 + 1; ++i) {
            if (i < 0 || i > n) continue;
            const double pv = x[2 * nv + static_cast<long long>(j) * np + i];
            gx = fma(sv::ccol(I, i) * sv::ncol(J, j), pv, gx);
            gy = fma(sv::ncol(I, i) * sv::ccol(J, j), pv, gy);
          }
        }
        ax = cl * sx + cb * gx;
        ay = cl * sy + cb * gy;
      }
      const double rx = b[k] - ax, ry = b[nv + k] - ay;
      acc = fma(rx, rx, acc);
      acc = fma(ry, ry, acc);
    }
  } else {
    const int j = r - nq;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
      double s = 0.0;
      for (int dJ = -2; dJ <= 2; ++dJ) {
        const int J = 2 * j + dJ;
        if (J <= 0 || J >= nq - 1) continue;
        for (int dI = -2; dI <= 2; ++dI) {
          const int I = 2 * i + dI;
          if (I <= 0 || I >= nq - 1) continue;
          const long long kk = static_cast<long long>(J) * nq + I;
          s = fma(sv::crow(dI) * sv::nrow(dJ), x[kk], s);
          s = fma(sv::nrow(dI) * sv::crow(dJ), x[nv + kk], s);
        }
      }
      const long long k = 2 * nv + static_cast<long long>(j) * np + i;
      const double rp = b[k] - cb * s;
      acc = fma(rp, rp, acc);
    }
  }
  const double t = na_block_sum(acc);
  if (threadIdx.x == 0) scratch[r] = t;
}

// norm = sqrt(sum of the rows' partials), summed in a fixed order by one CTA.
__global__ void k_resnorm_final(const double* __restrict__ scratch, int rows, double* __restrict__ norm) {
  sv::pdl_begin();
  double s = 0.0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) s += scratch[r];
  const double t = na_block_sum(s);
  if (threadIdx.x == 0) *norm = sqrt(t);
}

// ID of the current context (cuCtxGetId, through the runtime's driver entry
// points: unique for the life of the process, so a context created after a
// cudaDeviceReset never matches an entry of the one it replaced); 0 if unknown.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  if (!get_current || !get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || ctx == nullptr || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array in the current context of the current
// device (cudaGetSymbolAddress; host code cannot use the symbol itself), looked
// up once per device and context: a device reset (new context) looks it up again.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  // 0 before the device's context exists (the lookup below creates it): looked up again
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  ScratchEntry& ent = g_scratch[dev];
  if (ent.addr == nullptr || id == 0 || ent.ctx_id != id) {
    void* a = nullptr;
    e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    ent.addr = static_cast<double*>(a);
    ent.ctx_id = id;
  }
  *out = ent.addr;
  return cudaSuccess;
}

}  // namespace

extern "C" stokes_status stokes_residual_norm_noalloc(int n, double viscosity, const double* b,
                                                      const double* x, double* norm, void* stream) {
  if (n < 1 || n > STOKES_NOALLOC_MAX_N) {
    sv::set_last_error("stokes_residual_norm_noalloc: n must be in 1.." +
                       std::to_string(STOKES_NOALLOC_MAX_N) + " (size of its static scratch)");
    return STOKES_ERR_ARG;
  }
  if (!(viscosity > 0.0) || !std::isfinite(viscosity) || !b || !x || !norm) {
    sv::set_last_error("stokes_residual_norm_noalloc: viscosity must be > 0 and pointers non-null");
    return STOKES_ERR_ARG;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    sv::set_last_error(std::string("stokes_residual_norm_noalloc: scratch address: ") +
                       cudaGetErrorString(e));
    return STOKES_ERR_CUDA;
  }
  sv::LevelDev L{};   // fields this residual kernel does not use stay zero
  L.n = n;
  L.nq = 2 * n + 1;
  L.np = n + 1;
  L.nv = static_cast<long long>(L.nq) * L.nq;
  L.N = 2 * L.nv + static_cast<long long>(L.np) * L.np;
  L.h = 1.0 / n;
  L.nu = viscosity;
  L.cl = viscosity / 90.0;
  L.cb = -L.h / 18.0;
  L.clf = static_cast<float>(L.cl);
  L.cbf = static_cast<float>(L.cb);
  const int rows = L.nq + L.np;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  sv::launch_pdl(k_resnorm_rows, dim3(rows), dim3(256), 0, s, L, b, x, scratch);
  sv::launch_pdl(k_resnorm_final, dim3(1), dim3(1024), 0, s, scratch, rows, norm);
  sv::count_launches(2);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    sv::set_last_error(std::string("stokes_residual_norm_noalloc: launch: ") + cudaGetErrorString(e));
    return STOKES_ERR_CUDA;
  }
  return STOKES_OK;
}
