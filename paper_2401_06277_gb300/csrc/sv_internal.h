// sv_internal.h -- internal types of the Stokes/Vanka library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <utility>

#include <atomic>
#include <cstddef>
#include <string>
#include <vector>

#include "stokes_vanka.h"

namespace sv {

// ---- programmatic dependent launch (Hopper and later) ----
// Every kernel of the library begins with pdl_begin(), which waits until the
// previous kernel of the stream has completed with its memory operations
// visible; nothing is read or written before it.  A kernel started by
// launch_pdl may be launched once every CTA of its predecessor has exited
// (the implicit trigger), so its launch overlaps the predecessor's completion
// instead of following it; launched plainly, the wait returns at once.  There
// is no early trigger: dependents scheduled while their predecessor still
// runs would be placed unevenly over the SMs, which slows the kernels bound by
// the per-SM FP64 pipe.
__device__ __forceinline__ void pdl_begin() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);   // errors surface in cudaGetLastError
}


// Per-class patch data for the Schur-factored exact patch solve.  A patch
// matrix is A_i = [[K, 0, bx^T], [0, K, by^T], [bx, by, 0]] in slot order
// (u_x 5x5 window, u_y window, p); slots outside the domain or on Dirichlet
// nodes carry identity rows of K and zero b entries.  With z = K^-1 [bx by]^T
// and s = [bx by] z:  dp = (z . r_u - r_p) / s,  du = K^-1 r_u - z dp,
// which equals A_i^-1 r exactly (block elimination).
constexpr int CD_KINV = 0;      // 25 x 25, row-major (set-up only: kernels use the fast-diagonalisation factors)
constexpr int CD_Z = 625;       // 50: z for u_x slots, then u_y slots
constexpr int CD_SINV = 675;    // 1 / s
constexpr int CD_STRIDE = 680;  // doubles per class
constexpr int NCLASS = 25;
constexpr int INTERIOR_CLASS = 12;  // 5 * 2 + 2

// Fast diagonalisation of every class (appended to the class data at CD_EDGE).
// Per axis class a (vertex index 0, 1, interior, n-1, n) the free window slots
// F_a are {3,4}, {1..4}, {0..4}, {0..3}, {0,1}; on the free sub-rectangle
// F_ax x F_ay the block is K = (nu/90) (k_F (x) m_F + m_F (x) k_F) again, so
// K^-1 = (90/nu) (S_x (x) S_y) diag(1/(l_x + l_y)) (S_x (x) S_y)^T with the
// generalised eigenvectors k_F S = m_F S diag(l), S^T m_F S = I.  S is stored
// padded to 5 x 5 (zero rows off F_a, zero columns beyond |F_a|); slots off the
// free rectangle keep identity rows (Dirichlet nodes: correction = residual).
constexpr int EDGE_S = 0;        // 5 axis classes x [slot * 5 + mode]
constexpr int EDGE_DINV = 125;   // 25 classes x [mode_y * 5 + mode_x]: (90/nu) / (l_x + l_y), 0 if padded
constexpr int EDGE_TAB = 750;
constexpr int CD_EDGE = NCLASS * CD_STRIDE;
constexpr int CD_TOTAL = CD_EDGE + EDGE_TAB;   // doubles (or floats) of class data per level
// bit s set: window slot s of axis class a holds a free Q2 node
__host__ __device__ constexpr int axis_free_mask(int a) {
  return a == 0 ? 0x18 : a == 1 ? 0x1E : a == 2 ? 0x1F : a == 3 ? 0x0F : 0x03;
}

// Fast-diagonalisation factors of the interior patch block (see sv_setup.cu):
// se[m*3+k]: symmetric eigenvector k at reduced index m (entries 0/4, 1/3, 2);
// so[m*2+k]: antisymmetric eigenvector k at reduced index m (entries 0/-4, 1/-3);
// dinv[a*5+b] = (90/nu) / (l_a + l_b), eigenvalues ordered sym 0..2, anti 0..1.
// The solve's column pass (forward transform along y, division by l_a + l_b, inverse
// transform along y, for window column b) is one operator per column that keeps the
// parity split: gs[b*9 + m*3 + j] maps the symmetric inputs (v0 + v4, v1 + v3, v2)
// to the symmetric outputs m, ga[b*4 + m*2 + j] the antisymmetric (v0 - v4, v1 - v3):
//   gs = sum over sym modes a of se[m][a] dinv[a][b] se[j][a], ga likewise with so.
template <typename T>
struct FastDiagT {
  T se[9];
  T so[4];
  T dinv[25];
  T gs[45];
  T ga[20];
};
using FastDiag = FastDiagT<double>;

// A table in another arithmetic type, entry by entry (conv: S -> D).
template <typename D, typename S, typename F>
inline FastDiagT<D> fd_cast(const FastDiagT<S>& s, F conv) {
  FastDiagT<D> d;
  for (int k = 0; k < 9; ++k) d.se[k] = conv(s.se[k]);
  for (int k = 0; k < 4; ++k) d.so[k] = conv(s.so[k]);
  for (int k = 0; k < 25; ++k) d.dinv[k] = conv(s.dinv[k]);
  for (int k = 0; k < 45; ++k) d.gs[k] = conv(s.gs[k]);
  for (int k = 0; k < 20; ++k) d.ga[k] = conv(s.ga[k]);
  return d;
}

// Braess-Sarazin / Schur-Uzawa parameters (Sections 3.1, 3.3; see stokes_params).
constexpr int TC_WAIT_LIMIT = 1 << 22;   // polls of an mbarrier before a tensor-core sweep's wait gives up
constexpr int TAIL_SPIN_LIMIT = 1 << 22;   // polls (about 64 ns apart) of a grid barrier before it gives up


struct BSParams {
  double t = 1.0, omega = 1.0, jacobi_weight = 1.0;
  int jacobi_iters = 2;
  bool uzawa = false;   // Schur-Uzawa (Algorithm 4): no B^T dp in the velocity update
};

// Device-side description of one level (passed by value to kernels).
struct LevelDev {
  int n;       // elements per axis
  int nq;      // Q2 nodes per axis, 2n + 1
  int np;      // Q1 vertices per axis, n + 1
  long long nv;  // nq * nq
  long long N;   // 2 nv + np^2
  double h;    // 1 / n
  double nu;   // viscosity
  double cl;   // nu / 90: scale of the integer Laplacian stencil
  double cb;   // -h / 18: scale of the integer divergence stencil
  float clf, cbf;   // the same in FP32 (formed on the host: FP32 kernels do no FP64 arithmetic)
  // interior patches: z = K^-1 b^T = zs z_u with z_u the universal vector of the
  // integer stencils (interior_unit_schur), 1 / s = zsinv
  double zs, zsinv;
  float zsf, zsinvf;
};

// cl and cb in the element type
template <typename T>
__host__ __device__ inline T level_cl(const LevelDev& L);
template <>
__host__ __device__ inline double level_cl<double>(const LevelDev& L) { return L.cl; }
template <>
__host__ __device__ inline float level_cl<float>(const LevelDev& L) { return L.clf; }
template <typename T>
__host__ __device__ inline T level_cb(const LevelDev& L);
template <>
__host__ __device__ inline double level_cb<double>(const LevelDev& L) { return L.cb; }
template <>
__host__ __device__ inline float level_cb<float>(const LevelDev& L) { return L.cbf; }
template <typename T>
__host__ __device__ inline T level_zs(const LevelDev& L);
template <>
__host__ __device__ inline double level_zs<double>(const LevelDev& L) { return L.zs; }
template <>
__host__ __device__ inline float level_zs<float>(const LevelDev& L) { return L.zsf; }
template <typename T>
__host__ __device__ inline T level_zsinv(const LevelDev& L);
template <>
__host__ __device__ inline double level_zsinv<double>(const LevelDev& L) { return L.zsinv; }
template <>
__host__ __device__ inline float level_zsinv<float>(const LevelDev& L) { return L.zsinvf; }

// Persistent coarse-level kernel (sv_vanka.cu): the part of a V- or W-cycle
// (Algorithm 1) on the levels n <= stokes_params.tail_n of an FP32 preconditioner
// runs as one cooperative launch executing a list of steps separated by grid
// barriers.  The list is built on the host by walking the same recursion as the
// launch path, so both apply the same operations to the same buffers.
enum TailKind : int {
  TAIL_SWEEP = 0,     // c = sweep(level, x = a (null: zero guess), b)       (Algorithm 3)
  TAIL_ZERO = 1,      // c = 0 on level
  TAIL_RESID = 2,     // c = b - A a on level
  TAIL_RESTRICT = 3,  // c (level - 1) = P^T a (level)
  TAIL_PROLONG = 4,   // c (level) += P a (level - 1)
  TAIL_COARSE = 5,    // c = A_0^-1 a on level 0 (bordered inverse, FP64 arithmetic)
  TAIL_COPY = 6       // c = a on level
};
struct TailOp {
  int kind, level;
  const float* a;
  const float* b;
  float* c;
};
struct TailLevel {
  LevelDev d;
  const float* cd;    // FP32 class data of the level
};
constexpr int TAIL_NT = 128;   // threads per CTA (the 8 x 8 SIMT sweep tile)

struct Level {
  LevelDev d;
  double* x0 = nullptr;   // iterate (ping)
  double* x1 = nullptr;   // iterate (pong)
  double* b = nullptr;    // right-hand side of this level
  double* r = nullptr;    // residual scratch
  double* e = nullptr;    // V-cycle result of this level (coarse correction)
  double* cd = nullptr;   // NCLASS * CD_STRIDE class data (device)
  int vk_cfg = 0;         // tile shape of the FP64 sweep on this level
  // mixed-precision preconditioner (allocated when prec != STOKES_FP64)
  float* xf0 = nullptr;
  float* xf1 = nullptr;
  float* bf = nullptr;
  float* rf = nullptr;
  float* ef = nullptr;
  float* cdf = nullptr;   // class data in FP32
  int vk_cfg_f = 0;       // tile shape of the FP32 sweep on this level
  // tensor-core sweep (prec == STOKES_MIXED_BF16): interior tile range, BF16 inverse image
  int tc_lo = 1, tc_hi = 0;
  bool strip = false;     // the interior tiles [tc_lo, tc_hi]^2 have a strip sweep (both mixed forms)
  bool tc_on = true;      // the autotuner may prefer the SIMT sweep on small levels
  void* tcB = nullptr;    // BF16 form: the interior inverse for the tensor cores
  // simple Vanka (smoother == STOKES_SMOOTHER_PER_PATCH): per-patch inverses, entry-major
  double* pinv = nullptr;
  std::vector<double> cd_host;
  std::vector<double> full_inv_host;  // NCLASS * 51 * 51 dense inverses (host)
};

}  // namespace sv

struct stokes_hierarchy {
  stokes_params prm;
  double nu = 1.0;
  int n = 0;
  cudaStream_t stream = nullptr;
  std::vector<sv::Level> lv;     // lv[0] = coarsest
  sv::FastDiag fd;               // interior patch factors (level independent)
  sv::FastDiagT<float> fdf;      // the same in FP32
  double* coarse_G = nullptr;    // N0 x N0 dense inverse of the bordered coarse system
  int N0 = 0;
  // FGMRES workspace
  int m = 0;
  double* V = nullptr;           // (m + 1) x N
  double* Z = nullptr;           // m x N
  double* small = nullptr;       // H, g, cs, sn, hcol, h2, y, scalars
  double* partials = nullptr;    // dot-product partial sums
  int npart = 0;                 // blocks of the dot kernels
  unsigned* ticket = nullptr;    // last-block counter of the fused Gram-Schmidt kernels
  double* delta = nullptr;       // patch corrections of the simple-Vanka sweep (finest-level size)
  float* deltaf = nullptr;       // the same for the FP32 split sweep of the mixed forms
  void* bs_buf = nullptr;        // Braess-Sarazin scratch in the V-cycle precision (finest-level size)
  // block-triangular preconditioner: dense inverses of the coarsest L and M, 3 finest vectors
  double* bt_GL = nullptr;
  double* bt_GM = nullptr;
  int bt_nL = 0, bt_nM = 0;
  double* bt_buf = nullptr;
  sv::BSParams bs;
  double* host_scalars = nullptr;  // pinned host mirror of a few scalars
  int* dev_err = nullptr;          // set by kernels whose bounded waits expired
  int tc_wait_limit = sv::TC_WAIT_LIMIT;   // first bounded wait of the tensor-core sweep (test hook)
  // persistent coarse-level kernel (mixed forms): levels 0..tail_top in one launch
  int tail_top = -1;
  sv::TailOp* tail_ops = nullptr;      // device: the steps of one cycle below and at tail_top
  int tail_nops = 0;
  sv::TailLevel* tail_levels = nullptr;   // device: levels 0..tail_top
  unsigned* tail_bar = nullptr;        // device: grid-barrier count and generation
  int tail_grid = 0;                   // CTAs of the cooperative launch
  int tail_spin_limit = sv::TAIL_SPIN_LIMIT;
  int tail_skip_arrival = -1;          // test hook: this CTA withholds its first barrier arrival
  // BF16 form: the SIMT ring of boundary tiles runs on ring_stream while the
  // tensor-core kernel sweeps the interior tiles on stream (fork / join events)
  cudaStream_t ring_stream = nullptr;
  cudaEvent_t ring_fork = nullptr, ring_join = nullptr;
  double* aux = nullptr;           // finest-level vector: the projected adjoint right-hand side
  // measurement
  bool timing = false;
  long long vcycles = 0;
  std::vector<cudaEvent_t> ev_pool;   // pairs (start, stop) of finest-level sweeps
  size_t ev_used = 0;
  long long sweeps_timed = 0;
  double sweep_ms = 0.0;
};

namespace sv {

// FGMRES pieces (sv_api.cu): stream-ordered on h->stream, no host synchronisation.
// fg_scalars: device scalars sc[0] = ||V_0||^2 after fg_residual / fg_finish_cycle,
// sc[2] = residual estimate after fg_iteration.
double* fg_scalars(stokes_hierarchy* h);
void fg_residual(stokes_hierarchy* h, const double* b, const double* x);
void fg_start_cycle(stokes_hierarchy* h, double beta);
void fg_iteration(stokes_hierarchy* h, int j);
void fg_finish_cycle(stokes_hierarchy* h, int k, const double* b, double* x);

// message returned by stokes_last_error() on this thread
void set_last_error(const std::string& msg);

// kernels launched by this library (every launch_* adds its own count)
extern std::atomic<long long> g_launches;
extern std::atomic<long long> g_tc_launches;   // tensor-core sweep kernels among them
inline void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---- host setup (sv_setup.cu) ----
// Class data (Schur factors) for a level, and the 51 x 51 dense inverses.
void build_class_data(int n, double nu, std::vector<double>& cd, std::vector<double>* full_inv);
// The Schur data of an interior patch in the integer units of the stencils
// (Section 6.3: all interior patches share one matrix): z_u = K_u^-1 b_u^T with
// K_u = k (x) m + m (x) k and b_u = (C (x) N, N (x) C), s_u = b_u z_u.  A level
// scales them: z = (cb / cl) z_u, s = cb (cb / cl) s_u.
void interior_unit_schur(double* z50, double* s_unit);
// Uploads z_u to the constant memory of the Vanka sweep kernels (once per process).
cudaError_t set_interior_unit_z(const double* z50);
// Dense N0 x N0 operator of a level (Dirichlet-eliminated), row-major.
void dense_operator(int n, double nu, std::vector<double>& A);
// G = leading N0 x N0 block of [[A, e], [e^T, 0]]^-1, e = (0, M_p 1).
bool coarse_inverse(int n, double nu, std::vector<double>& G);
// Interior-class fast-diagonalisation factors (level independent for constant nu).
FastDiag interior_fast_diag(double nu);
// The EDGE_TAB fast-diagonalisation table of every class (layout above).
void edge_fast_diag(double nu, double* tab);
// In-place Gauss-Jordan inverse with partial pivoting; false if singular.
bool invert_dense(std::vector<double>& a, int m);

// ---- stencil kernels (sv_kernels.cu; T = double or float) ----
template <typename T>
void launch_apply(const LevelDev& L, const T* x, const T* b, T* y, int residual, cudaStream_t s);
void launch_rhs(const LevelDev& L, const double* f, const double* ud, double* b, cudaStream_t s);
void launch_rhs_transpose(const LevelDev& L, const double* lam, double* g, cudaStream_t s);
// Fused Vanka sweep (sv_vanka.cu, R = double or float); cfg selects the tile
// shape (8x8, 16x8, 16x16, 14x14 vertices).  Tiles (bx, by) with both indices
// in [skip_lo, skip_hi] are left to the tensor-core kernel (empty by default).
constexpr int VANKA_NCFG = 4;
constexpr int VANKA_CFG_14 = 3;
constexpr int VANKA_CFG_SPLIT = 4;   // FP64 only: own-patch solves + separate update (launch_vanka_split)
constexpr int VANKA_CFG_SPLIT2 = 5;  // the same, compiled for two CTAs per SM (at most 128 registers)
constexpr int VANKA_CFG_4 = 6;       // fused 4x4 tiles: small levels, spread over more SMs
inline bool vanka_cfg_split(int cfg) { return cfg == VANKA_CFG_SPLIT || cfg == VANKA_CFG_SPLIT2; }
template <typename R>
void launch_vanka(const LevelDev& L, const R* cd, const FastDiagT<R>& fd, const R* x, const R* b, R* xo,
                  double omega, int cfg, cudaStream_t s, int skip_lo = 1, int skip_hi = 0);

// Persistent coarse-level kernel (sv_vanka.cu): one cooperative launch of `grid`
// CTAs runs the nops steps; err is set to 1 if a grid barrier gave up.
cudaError_t tail_prepare(int* max_ctas);
void launch_tail(const TailOp* ops, int nops, const TailLevel* levels, const double* G, int N0,
                 const FastDiagT<float>& fd, double omega, unsigned* bar, int* err, int spin_limit,
                 int skip_arrival, int grid, cudaStream_t s);

// Tensor-core sweep (sv_vanka_tc.cu, FP32 vectors, BF16 tcgen05 patch GEMM):
// sweeps the 14 x 14 tiles [lo, hi]^2 whose patches are all of the interior
// class; the remaining tiles go to launch_vanka<float> with cfg 14x14 and
// skip range [lo, hi].  Bcanon: the interior inverse, 64 x 64 BF16 in the
// core-matrix layout (8 KB).  err: set to 1 if a bounded device wait expired.
constexpr int TC_TILE = 14;
void tc_interior_range(int n, int* lo, int* hi);
// first_wait_limit: polls of the wait for the inverse's bulk copy (0: it expires
// at once -- a test hook; the kernel then reports through *err and still waits
// for its copy with the full limit before it exits)
void launch_vanka_tc(const LevelDev& L, const void* Bcanon, const float* x, const float* b, float* xo,
                     double omega, int lo, int hi, int* err, cudaStream_t s, int first_wait_limit = TC_WAIT_LIMIT);
cudaError_t vanka_tc_prepare();
// The FP32 strip sweep of the same interior tiles (mixed FP32 form): the strip walk
// of launch_vanka_tc with every patch solved exactly in FP32 by fast
// diagonalisation (fd: the interior factors) instead of the BF16 GEMM.
void launch_vanka_strip_f32(const LevelDev& L, const FastDiagT<float>& fd, const float* x, const float* b,
                            float* xo, double omega, int lo, int hi, cudaStream_t s);
// uploads z_u (50 doubles, as for set_interior_unit_z) for the FP32 strip sweep
cudaError_t set_strip_unit_z(const double* z50);
// 64 x 64 BF16 core-matrix image (uint16 bits) of a 51 x 51 row-major inverse
void tc_pack_inverse(const double* inv51, unsigned short* out4096);
const char* vanka_cfg_name(int cfg);
template <typename T>
void launch_restrict(const LevelDev& F, const LevelDev& C, const T* rf, T* rc, cudaStream_t s);
template <typename T>
void launch_prolong_add(const LevelDev& F, const LevelDev& C, const T* ec, T* xf, cudaStream_t s);
template <typename TI, typename TO>
void launch_convert(const TI* in, TO* out, long long N, cudaStream_t s);
void launch_coarse(const double* G, int N0, const double* r, double* e, cudaStream_t s);
cudaError_t vanka_prepare();

// ---- Braess-Sarazin relaxation (sv_bs.cu) ----
size_t bs_scratch_elems(const LevelDev& L);   // 2 nv + 3 np^2
// x_out = x + omega (du, dp) (Algorithm 2); x may be nullptr (zero guess);
// rbuf (level size) receives b - A x; scratch holds bs_scratch_elems(L)
template <typename T>
void launch_bs_sweep(const LevelDev& L, const BSParams& prm, T* scratch, T* rbuf, const T* x, const T* b, T* xo,
                     cudaStream_t s);

// ---- block-triangular preconditioner kernels (sv_bt.cu), FP64 ----
// y_p = b_p - M x_p (x may be nullptr), y_u = 0
void launch_mass_resid(const LevelDev& L, const double* x, const double* b, double* y, cudaStream_t s);
// xo = x + omega D^-1 r on block (0 velocity / diag L, 1 pressure / diag M), 0 on the other
void launch_block_jacobi(const LevelDev& L, int block, const double* x, const double* r, double* xo, double omega,
                         cudaStream_t s);
void launch_add(double* y, const double* x, long long N, cudaStream_t s);   // y += x
// host: dense inverses of the coarsest velocity Laplacian block and pressure mass matrix
bool bt_coarse_inverses(int n, double nu, std::vector<double>& GL, std::vector<double>& GM);

// ---- simple Vanka (sv_simple.cu): per-patch inverses, FP64 ----
int patch_stride(const LevelDev& L);                 // patch count rounded up to 32
size_t patch_inverse_doubles(const LevelDev& L);     // 51 * 51 * stride
size_t patch_delta_doubles(const LevelDev& L);       // 51 * stride
// scratch of the split sweep (launch_vanka_split): per-patch corrections of its edge
// tiles, the column sums of every tile and the pressure corrections
size_t split_delta_doubles(const LevelDev& L);
cudaError_t simple_prepare();
void launch_patch_inverse(const LevelDev& L, double* inv, cudaStream_t s);
// xo = x + sum_i V_i^T W_i A_i^-1 V_i (b - A x) with the stored inverses; x may
// be nullptr (zero guess); rscratch (level size) receives b - A x; delta
// (patch_delta_doubles) the corrections
// x_out = x + sum over patches of (omega / m_j) delta (entry-major corrections, stride P)
template <typename T>
void launch_patch_update(const LevelDev& L, int P, const T* delta, const T* x, T* xo, double omega, cudaStream_t s);
// Split sweep: own-patch solves (16 x 16 tiles, no halo patches) writing column
// sums of the corrections into delta (split_delta_doubles), then the update.
// rscratch (may be null): a level vector that receives r = b - A x first, so the
// residual is formed once per cell instead of on the tiles' halo.
template <typename R>
void launch_vanka_split(const LevelDev& L, const R* cd, const FastDiagT<R>& fd, const R* x, const R* b, R* xo,
                        double omega, R* delta, int two_per_sm, cudaStream_t s, R* rscratch);
void launch_simple_sweep(const LevelDev& L, const double* inv, double* delta, double* rscratch, const double* x,
                         const double* b, double* xo, double omega, cudaStream_t s);

// ---- Krylov kernels (sv_krylov.cu) ----
int dot_blocks();
// Gram-Schmidt pass 1 over V_k = V + k * ld, k < nk: dots[k] = <V_k, w>; if
// norm2 != nullptr also norm2[0] = <w, w>, norm2[1] = sqrt(norm2[0]).  Does
// nothing when gate != nullptr and *gate == 0.  partials holds
// (ORTH_KMAX + 1) * npart doubles; ticket is a zeroed device counter, reset
// by each launch before it ends (one stream at a time per ticket).
void launch_orth_dots(const double* V, long long ld, int nk, const double* w, long long N, double* partials,
                      int npart, unsigned* ticket, double* dots, double* norm2, const double* gate,
                      cudaStream_t s);
// Gram-Schmidt pass 2: w -= sum_k coef[k] V_k; norm2 as above for the updated
// w; if dgks_ref != nullptr, *flag = (norm2[0] < *dgks_ref / 2) as 1.0 / 0.0;
// if hacc != nullptr, hacc[k] += coef[k] for k < nk.  Gated like pass 1.
void launch_orth_update(double* w, const double* V, long long ld, int nk, const double* coef, long long N,
                        double* partials, int npart, unsigned* ticket, double* norm2, const double* gate,
                        const double* dgks_ref, double* flag, double* hacc, cudaStream_t s);
// Pass 1's update and pass 2's dots in one launch (see k_orth_update_dots);
// returns false, launching nothing, when nk is outside 1..16.
bool launch_orth_update_dots(double* w, const double* V, long long ld, int nk, const double* coef, long long N,
                             double* partials, int npart, unsigned* ticket, double* dots, double* norm2,
                             const double* dgks_ref, double* flag, cudaStream_t s);
// One step of modified Gram-Schmidt (see k_mgs_step): w -= coef[0] Va unless Va
// is null; dots[0] = <Vb, w> unless Vb is null; when Va or Vb is null also
// norm2[0] = <w, w>, norm2[1] = its root (first step: of w as given; last step:
// of the updated w).  Va and Vb are not both null.  partials and ticket as for
// launch_orth_dots.
void launch_mgs_step(double* w, const double* Va, const double* Vb, const double* coef, long long N,
                     double* partials, int npart, unsigned* ticket, double* dots, double* norm2, cudaStream_t s);
// w += sign * sum_k coef[k] V_k
void launch_multiaxpy(double* w, const double* V, long long ld, int nk, const double* coef,
                      double sign, long long N, cudaStream_t s);
// y = x * (1 / *den) (den on device; y = 0 if *den == 0) ; or y = x * scal if den == nullptr
void launch_scale(double* y, const double* x, const double* den, double scal, long long N,
                  cudaStream_t s);
// Givens step for column j of H (ld = m + 1); writes |g[j+1]| to *est
void launch_givens(double* H, int ldh, double* cs, double* sn, double* g, const double* hcol,
                   const double* hnorm, int j, double* est, cudaStream_t s);
void launch_backsolve(const double* H, int ldh, const double* g, int k, double* y, cudaStream_t s);
void launch_fill(double* p, double v, long long N, cudaStream_t s);
// y = x with its pressure block shifted to zero (Euclidean) mean: the component
// of x along ker A^T = (0, 1_p) is removed, so y is a consistent right-hand side
void launch_project_pressure(const LevelDev& L, const double* x, double* y, double* partials, int npart,
                             double* sum, cudaStream_t s);
// dst = src on Dirichlet velocity rows, 0 elsewhere
void launch_dirichlet_copy(const LevelDev& L, const double* src, double* dst, cudaStream_t s);

}  // namespace sv
