// sv_setup.cu -- host-side set-up of one level: the 25 Vanka patch-class
// factorisations (Section 6.3: on a uniform grid the patch matrices
// A_i = V_i A V_i^T take only 25 distinct values) and the exact coarse-grid
// inverse (Algorithm 1, level 0).  Plain FP64, run once per hierarchy.
#include <cmath>
#include <vector>

#include "sv_internal.h"
#include "sv_stencil.cuh"

namespace sv {

bool invert_dense(std::vector<double>& a, int m) {
  std::vector<double> inv(static_cast<size_t>(m) * m, 0.0);
  for (int i = 0; i < m; ++i) inv[static_cast<size_t>(i) * m + i] = 1.0;
  for (int col = 0; col < m; ++col) {
    int piv = col;
    double best = std::fabs(a[static_cast<size_t>(col) * m + col]);
    for (int r = col + 1; r < m; ++r) {
      double v = std::fabs(a[static_cast<size_t>(r) * m + col]);
      if (v > best) { best = v; piv = r; }
    }
    if (!(best > 0.0)) return false;
    if (piv != col) {
      for (int k = 0; k < m; ++k) {
        std::swap(a[static_cast<size_t>(piv) * m + k], a[static_cast<size_t>(col) * m + k]);
        std::swap(inv[static_cast<size_t>(piv) * m + k], inv[static_cast<size_t>(col) * m + k]);
      }
    }
    double d = 1.0 / a[static_cast<size_t>(col) * m + col];
    for (int k = 0; k < m; ++k) {
      a[static_cast<size_t>(col) * m + k] *= d;
      inv[static_cast<size_t>(col) * m + k] *= d;
    }
    for (int r = 0; r < m; ++r) {
      if (r == col) continue;
      double f = a[static_cast<size_t>(r) * m + col];
      if (f == 0.0) continue;
      for (int k = 0; k < m; ++k) {
        a[static_cast<size_t>(r) * m + k] -= f * a[static_cast<size_t>(col) * m + k];
        inv[static_cast<size_t>(r) * m + k] -= f * inv[static_cast<size_t>(col) * m + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

namespace {

// Representative vertex index of a per-axis class on an n x n grid.
int class_rep(int c, int n) {
  switch (c) {
    case 0: return 0;
    case 1: return 1;
    case 2: return 2;
    case 3: return n - 1;
    default: return n;
  }
}

bool free_node(int I, int J, int nq) { return I > 0 && J > 0 && I < nq - 1 && J < nq - 1; }
bool in_grid(int I, int J, int nq) { return I >= 0 && J >= 0 && I < nq && J < nq; }

// Entry of the scalar block nu*(K (x) M + M (x) K) between Q2 nodes (I,J) and (I2,J2).
double lap_entry(int I, int J, int I2, int J2, double nu) {
  int dI = I2 - I, dJ = J2 - J;
  if (dI < -2 || dI > 2 || dJ < -2 || dJ > 2) return 0.0;
  return nu / 90.0 * (k1(I, dI) * m1(J, dJ) + m1(I, dI) * k1(J, dJ));
}

}  // namespace

void build_class_data(int n, double nu, std::vector<double>& cd, std::vector<double>* full_inv) {
  const int nq = 2 * n + 1;
  const double h = 1.0 / n;
  cd.assign(static_cast<size_t>(NCLASS) * CD_STRIDE, 0.0);
  if (full_inv) full_inv->assign(static_cast<size_t>(NCLASS) * 51 * 51, 0.0);
  for (int cy = 0; cy < 5; ++cy) {
    for (int cx = 0; cx < 5; ++cx) {
      const int cls = 5 * cy + cx;
      const int pi = class_rep(cx, n), pj = class_rep(cy, n);
      // K (25 x 25) on the window nodes; identity on Dirichlet / outside slots
      std::vector<double> K(625, 0.0);
      bool act[25];
      int nI[25], nJ[25];
      for (int s = 0; s < 25; ++s) {
        nI[s] = 2 * pi + (s % 5) - 2;
        nJ[s] = 2 * pj + (s / 5) - 2;
        act[s] = in_grid(nI[s], nJ[s], nq) && free_node(nI[s], nJ[s], nq);
      }
      for (int s = 0; s < 25; ++s) {
        for (int t = 0; t < 25; ++t) {
          double v;
          if (!act[s] || !act[t]) v = (s == t && !act[s]) ? 1.0 : 0.0;
          else v = lap_entry(nI[s], nJ[s], nI[t], nJ[t], nu);
          K[s * 25 + t] = v;
        }
      }
      // B row of the patch pressure (vertex (pi, pj)): b(v,p) = -int p div v
      double bx[25], by[25];
      for (int s = 0; s < 25; ++s) {
        int dI = nI[s] - 2 * pi, dJ = nJ[s] - 2 * pj;
        bx[s] = act[s] ? -h / 18.0 * crow(dI) * nrow(dJ) : 0.0;
        by[s] = act[s] ? -h / 18.0 * nrow(dI) * crow(dJ) : 0.0;
      }
      std::vector<double> Kinv = K;
      invert_dense(Kinv, 25);
      double* C = cd.data() + static_cast<size_t>(cls) * CD_STRIDE;
      for (int k = 0; k < 625; ++k) C[CD_KINV + k] = Kinv[k];
      double s = 0.0;
      for (int o = 0; o < 25; ++o) {
        double zx = 0.0, zy = 0.0;
        for (int k = 0; k < 25; ++k) {
          zx += Kinv[o * 25 + k] * bx[k];
          zy += Kinv[o * 25 + k] * by[k];
        }
        C[CD_Z + o] = zx;
        C[CD_Z + 25 + o] = zy;
      }
      for (int k = 0; k < 25; ++k) s += bx[k] * C[CD_Z + k] + by[k] * C[CD_Z + 25 + k];
      C[CD_SINV] = 1.0 / s;
      if (full_inv) {
        // A_i^-1 = [[K^-1 - z z^T / s, z / s], [z^T / s, -1 / s]] (block elimination)
        double* F = full_inv->data() + static_cast<size_t>(cls) * 51 * 51;
        const double* z = C + CD_Z;
        for (int a = 0; a < 50; ++a) {
          for (int c = 0; c < 50; ++c) {
            double kin = ((a < 25) == (c < 25)) ? Kinv[(a % 25) * 25 + (c % 25)] : 0.0;
            F[a * 51 + c] = kin - z[a] * z[c] / s;
          }
          F[a * 51 + 50] = z[a] / s;
          F[50 * 51 + a] = z[a] / s;
        }
        F[50 * 51 + 50] = -1.0 / s;
      }
    }
  }
}

void dense_operator(int n, double nu, std::vector<double>& A) {
  const int nq = 2 * n + 1, np = n + 1;
  const long long nv = static_cast<long long>(nq) * nq;
  const long long N = 2 * nv + static_cast<long long>(np) * np;
  const double h = 1.0 / n;
  A.assign(static_cast<size_t>(N * N), 0.0);
  auto at = [&](long long r, long long c) -> double& { return A[static_cast<size_t>(r * N + c)]; };
  for (int J = 0; J < nq; ++J) {
    for (int I = 0; I < nq; ++I) {
      long long kx = static_cast<long long>(J) * nq + I, ky = nv + kx;
      if (!free_node(I, J, nq)) {
        at(kx, kx) = 1.0;
        at(ky, ky) = 1.0;
        continue;
      }
      for (int J2 = J - 2; J2 <= J + 2; ++J2) {
        for (int I2 = I - 2; I2 <= I + 2; ++I2) {
          if (!in_grid(I2, J2, nq) || !free_node(I2, J2, nq)) continue;
          double v = lap_entry(I, J, I2, J2, nu);
          long long c = static_cast<long long>(J2) * nq + I2;
          at(kx, c) += v;
          at(ky, nv + c) += v;
        }
      }
      for (int j = J / 2 - 1; j <= J / 2 + 1; ++j) {
        for (int i = I / 2 - 1; i <= I / 2 + 1; ++i) {
          if (i < 0 || j < 0 || i > n || j > n) continue;
          long long c = 2 * nv + static_cast<long long>(j) * np + i;
          at(kx, c) += -h / 18.0 * ccol(I, i) * ncol(J, j);
          at(ky, c) += -h / 18.0 * ncol(I, i) * ccol(J, j);
        }
      }
    }
  }
  for (int j = 0; j < np; ++j) {
    for (int i = 0; i < np; ++i) {
      long long kp = 2 * nv + static_cast<long long>(j) * np + i;
      for (int dJ = -2; dJ <= 2; ++dJ) {
        for (int dI = -2; dI <= 2; ++dI) {
          int I = 2 * i + dI, J = 2 * j + dJ;
          if (!in_grid(I, J, nq) || !free_node(I, J, nq)) continue;
          long long c = static_cast<long long>(J) * nq + I;
          at(kp, c) += -h / 18.0 * crow(dI) * nrow(dJ);
          at(kp, nv + c) += -h / 18.0 * nrow(dI) * crow(dJ);
        }
      }
    }
  }
}

bool coarse_inverse(int n, double nu, std::vector<double>& G) {
  std::vector<double> A;
  dense_operator(n, nu, A);
  const int nq = 2 * n + 1, np = n + 1;
  const long long nv = static_cast<long long>(nq) * nq;
  const int N = static_cast<int>(2 * nv + np * np);
  const int M = N + 1;
  const double h = 1.0 / n;
  std::vector<double> Kb(static_cast<size_t>(M) * M, 0.0);
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < N; ++c) Kb[static_cast<size_t>(r) * M + c] = A[static_cast<size_t>(r) * N + c];
  // e_p = M_p 1 = int phi_k: h^2 times 1 (interior), 1/2 (edge), 1/4 (corner)
  for (int j = 0; j < np; ++j) {
    for (int i = 0; i < np; ++i) {
      double wi = (i == 0 || i == n) ? 0.5 : 1.0, wj = (j == 0 || j == n) ? 0.5 : 1.0;
      int k = static_cast<int>(2 * nv) + j * np + i;
      Kb[static_cast<size_t>(k) * M + N] = h * h * wi * wj;
      Kb[static_cast<size_t>(N) * M + k] = h * h * wi * wj;
    }
  }
  if (!invert_dense(Kb, M)) return false;
  G.assign(static_cast<size_t>(N) * N, 0.0);
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < N; ++c) G[static_cast<size_t>(r) * N + c] = Kb[static_cast<size_t>(r) * M + c];
  return true;
}

}  // namespace sv
