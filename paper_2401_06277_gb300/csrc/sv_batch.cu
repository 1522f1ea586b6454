// sv_batch.cu -- many independent Stokes problems (same or different grid
// sizes) solved together: right-preconditioned FGMRES (Section 6.8) in
// lockstep over the problems, with iteration j of every problem -- its V-cycle
// (Algorithm 1 with additive Vanka, Algorithm 3), operator, Gram-Schmidt Arnoldi and
// Givens rotation -- recorded once as a CUDA graph with one branch per
// problem.  Branches are independent, so the GPU runs the many small
// coarse-level kernels of all problems concurrently; the host synchronises
// once per iteration to read every problem's residual estimate.
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "sv_internal.h"

struct stokes_batch {
  std::vector<stokes_hierarchy*> hs;
  cudaStream_t caller = nullptr;         // stream given at creation (synchronised on entry)
  cudaStream_t main = nullptr;           // capture / graph-launch stream
  std::vector<cudaStream_t> side;        // one stream per problem
  std::vector<cudaEvent_t> join;         // one event per problem
  cudaEvent_t fork = nullptr;
  int m = 0;
  std::vector<cudaGraphExec_t> exec;     // exec[j]: iteration j of the captured problems
  std::vector<int> captured;             // problems in the captured graphs
  double* host = nullptr;                // pinned: one scalar per problem
};

namespace {

void destroy_graphs(stokes_batch* b) {
  for (cudaGraphExec_t g : b->exec)
    if (g) cudaGraphExecDestroy(g);
  b->exec.clear();
  b->captured.clear();
}

void destroy_batch(stokes_batch* b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  for (cudaStream_t s : b->side)
    if (s) cudaStreamSynchronize(s);
  destroy_graphs(b);
  for (stokes_hierarchy* h : b->hs)
    if (h) stokes_hierarchy_destroy(h);
  for (cudaStream_t s : b->side)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->main) cudaStreamDestroy(b->main);
  if (b->host) cudaFreeHost(b->host);
  delete b;
}

stokes_status batch_fail(stokes_status st, const std::string& msg) {
  sv::set_last_error(msg);
  return st;
}

// Record iterations 0..m-1 of the problems in `act` as m CUDA graphs.
cudaError_t capture(stokes_batch* b, const std::vector<int>& act) {
  destroy_graphs(b);
  b->exec.assign(b->m, nullptr);
  for (int j = 0; j < b->m; ++j) {
    cudaError_t e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaEventRecord(b->fork, b->main);
    for (int k : act) {
      stokes_hierarchy* h = b->hs[k];
      cudaStreamWaitEvent(b->side[k], b->fork, 0);
      sv::fg_iteration(h, j);
      cudaMemcpyAsync(b->host + k, sv::fg_scalars(h) + 2, sizeof(double), cudaMemcpyDeviceToHost, b->side[k]);
      cudaEventRecord(b->join[k], b->side[k]);
      cudaStreamWaitEvent(b->main, b->join[k], 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->main, &g);
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&b->exec[j], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
  }
  b->captured = act;
  return cudaGetLastError();
}

// main waits for the side streams of `act`
void join_all(stokes_batch* b, const std::vector<int>& act) {
  for (int k : act) {
    cudaEventRecord(b->join[k], b->side[k]);
    cudaStreamWaitEvent(b->main, b->join[k], 0);
  }
}

// copy sc[0] (= ||V_0||^2) of every problem in `act` to b->host and synchronise
cudaError_t read_norms(stokes_batch* b, const std::vector<int>& act) {
  for (int k : act)
    cudaMemcpyAsync(b->host + k, sv::fg_scalars(b->hs[k]), sizeof(double), cudaMemcpyDeviceToHost,
                    b->side[k]);
  for (int k : act) {
    cudaError_t e = cudaStreamSynchronize(b->side[k]);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

int device_error(stokes_batch* b) {
  int flag = 0;
  for (stokes_hierarchy* h : b->hs) {
    int f = 0;
    if (cudaMemcpy(&f, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && f) flag = 1;
  }
  return flag;
}

}  // namespace

extern "C" {

stokes_status stokes_batch_create(int nprob, const int* n, double viscosity, const stokes_params* params,
                                  void* stream, stokes_batch** out) {
  if (!out || nprob < 1 || !n) return batch_fail(STOKES_ERR_ARG, "stokes_batch_create: bad argument");
  *out = nullptr;
  stokes_params prm;
  stokes_default_params(&prm);
  if (params) prm = *params;
  auto* b = new (std::nothrow) stokes_batch();
  if (!b) return batch_fail(STOKES_ERR_OOM, "host allocation failed");
  b->caller = static_cast<cudaStream_t>(stream);
  b->m = prm.restart;
  cudaError_t e = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&b->host), nprob * sizeof(double));
  if (e != cudaSuccess) {
    destroy_batch(b);
    return batch_fail(e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA,
                      std::string("stokes_batch_create: ") + cudaGetErrorString(e));
  }
  b->side.assign(nprob, nullptr);
  b->join.assign(nprob, nullptr);
  b->hs.assign(nprob, nullptr);
  std::map<int, int> first;  // grid size -> first problem of that size (its tiles are reused)
  for (int k = 0; k < nprob; ++k) {
    if ((e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming)) != cudaSuccess) {
      destroy_batch(b);
      return batch_fail(STOKES_ERR_CUDA, std::string("stokes_batch_create: ") + cudaGetErrorString(e));
    }
    stokes_params pk = prm;
    auto it = first.find(n[k]);
    if (it != first.end() && prm.tile < 0) pk.tile = 0;  // tuned once per size, copied below
    stokes_status st = stokes_hierarchy_create(n[k], viscosity, &pk, b->side[k], &b->hs[k]);
    if (st != STOKES_OK) {
      destroy_batch(b);
      return st;
    }
    if (it == first.end()) {
      first[n[k]] = k;
    } else if (prm.tile < 0) {
      stokes_hierarchy* ref = b->hs[it->second];
      for (size_t l = 0; l < ref->lv.size(); ++l) {
        b->hs[k]->lv[l].vk_cfg = ref->lv[l].vk_cfg;
        b->hs[k]->lv[l].vk_cfg_f = ref->lv[l].vk_cfg_f;
        b->hs[k]->lv[l].tc_on = ref->lv[l].tc_on;
      }
    }
  }
  *out = b;
  return STOKES_OK;
}

stokes_status stokes_batch_destroy(stokes_batch* b) {
  destroy_batch(b);
  return STOKES_OK;
}

stokes_status stokes_batch_hierarchy(stokes_batch* b, int k, stokes_hierarchy** out) {
  if (!b || !out || k < 0 || k >= static_cast<int>(b->hs.size()))
    return batch_fail(STOKES_ERR_ARG, "stokes_batch_hierarchy: bad argument");
  *out = b->hs[k];
  return STOKES_OK;
}

stokes_status stokes_batch_solve(stokes_batch* b, const double* const* rhs, double* const* x, int* iters,
                                 double* relres) {
  if (!b || !rhs || !x) return batch_fail(STOKES_ERR_ARG, "stokes_batch_solve: null argument");
  const int P = static_cast<int>(b->hs.size());
  for (int k = 0; k < P; ++k)
    if (!rhs[k] || !x[k] || rhs[k] == x[k]) return batch_fail(STOKES_ERR_ARG, "stokes_batch_solve: bad vector");
  cudaError_t e = cudaStreamSynchronize(b->caller);  // inputs produced on the caller's stream
  if (e != cudaSuccess) return batch_fail(STOKES_ERR_CUDA, cudaGetErrorString(e));
  std::vector<double> beta0(P, 0.0), beta(P, 0.0), tol(P, 0.0);
  std::vector<int> it_k(P, 0), kk(P, 0);
  std::vector<char> done(P, 0), hit(P, 0);
  std::vector<int> all(P);
  for (int k = 0; k < P; ++k) all[k] = k;
  for (int k = 0; k < P; ++k) sv::fg_residual(b->hs[k], rhs[k], x[k]);
  if ((e = read_norms(b, all)) != cudaSuccess) return batch_fail(STOKES_ERR_CUDA, cudaGetErrorString(e));
  std::vector<int> act;
  for (int k = 0; k < P; ++k) {
    beta0[k] = beta[k] = std::sqrt(b->host[k]);
    if (!std::isfinite(beta0[k])) return batch_fail(STOKES_ERR_NONFINITE, "initial residual is not finite");
    tol[k] = b->hs[k]->prm.rtol * beta0[k];
    if (beta0[k] == 0.0) done[k] = 1;
    else act.push_back(k);
  }
  int it = 0;
  const int maxit = b->hs[0]->prm.maxit;
  while (!act.empty() && it < maxit) {
    for (int k : act) {
      sv::fg_start_cycle(b->hs[k], beta[k]);
      hit[k] = 0;
      kk[k] = 0;
    }
    if (b->captured != act) {
      if ((e = capture(b, act)) != cudaSuccess)
        return batch_fail(STOKES_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    join_all(b, act);
    for (int j = 0; j < b->m; ++j) {
      if ((e = cudaGraphLaunch(b->exec[j], b->main)) != cudaSuccess ||
          (e = cudaStreamSynchronize(b->main)) != cudaSuccess)
        return batch_fail(STOKES_ERR_CUDA, std::string("iteration graph: ") + cudaGetErrorString(e));
      ++it;
      bool all_hit = true;
      for (int k : act) {
        if (hit[k]) continue;
        const double est = b->host[k];
        if (!std::isfinite(est)) return batch_fail(STOKES_ERR_NONFINITE, "residual estimate is not finite");
        kk[k] = j + 1;
        if (est <= tol[k]) {
          hit[k] = 1;
          it_k[k] = it;
        } else {
          all_hit = false;
        }
      }
      if (all_hit || it >= maxit) break;
    }
    // the side streams continue after the graphs (the rest of the cycle runs on them)
    for (int k : act) {
      cudaEventRecord(b->join[k], b->main);
      cudaStreamWaitEvent(b->side[k], b->join[k], 0);
      sv::fg_finish_cycle(b->hs[k], kk[k], rhs[k], x[k]);
    }
    if ((e = read_norms(b, act)) != cudaSuccess) return batch_fail(STOKES_ERR_CUDA, cudaGetErrorString(e));
    std::vector<int> next;
    for (int k : act) {
      beta[k] = std::sqrt(b->host[k]);
      if (!std::isfinite(beta[k])) return batch_fail(STOKES_ERR_NONFINITE, "residual is not finite");
      if (!hit[k]) it_k[k] = it;
      if (beta[k] <= tol[k]) done[k] = 1;
      else next.push_back(k);
    }
    act.swap(next);
  }
  if (device_error(b)) return batch_fail(STOKES_ERR_TIMEOUT, "a bounded device wait expired");
  bool all_done = true;
  for (int k = 0; k < P; ++k) {
    if (iters) iters[k] = it_k[k];
    if (relres) relres[k] = beta0[k] > 0.0 ? beta[k] / beta0[k] : 0.0;
    if (!done[k]) all_done = false;
  }
  if (!all_done) return batch_fail(STOKES_NOT_CONVERGED, "FGMRES reached maxit for some problems");
  return STOKES_OK;
}

}  // extern "C"
