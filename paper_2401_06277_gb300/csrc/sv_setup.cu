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

void interior_unit_schur(double* z50, double* s_unit) {
  // slot s of the window: offset (s % 5 - 2, s / 5 - 2) from the vertex node, whose
  // coordinates are even, so the node parities are those of s % 5 and s / 5
  std::vector<double> K(625, 0.0);
  for (int a = 0; a < 25; ++a)
    for (int t = 0; t < 25; ++t) {
      const int PI = (a % 5) & 1, PJ = (a / 5) & 1, dI = t % 5 - a % 5, dJ = t / 5 - a / 5;
      K[a * 25 + t] = k1(PI, dI) * m1(PJ, dJ) + m1(PI, dI) * k1(PJ, dJ);
    }
  invert_dense(K, 25);
  double sum = 0.0;
  for (int o = 0; o < 25; ++o) {
    double zx = 0.0, zy = 0.0;
    for (int k = 0; k < 25; ++k) {
      const int dI = k % 5 - 2, dJ = k / 5 - 2;
      zx += K[o * 25 + k] * (crow(dI) * nrow(dJ));
      zy += K[o * 25 + k] * (nrow(dI) * crow(dJ));
    }
    z50[o] = zx;
    z50[25 + o] = zy;
  }
  for (int k = 0; k < 25; ++k) {
    const int dI = k % 5 - 2, dJ = k / 5 - 2;
    sum += crow(dI) * nrow(dJ) * z50[k] + nrow(dI) * crow(dJ) * z50[25 + k];
  }
  *s_unit = sum;
}

void build_class_data(int n, double nu, std::vector<double>& cd, std::vector<double>* full_inv) {
  const int nq = 2 * n + 1;
  const double h = 1.0 / n;
  cd.assign(static_cast<size_t>(CD_TOTAL), 0.0);
  edge_fast_diag(nu, cd.data() + CD_EDGE);
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

// ---------------------------------------------------------------------------
// Fast diagonalisation of the interior patch block.  On an interior patch the
// velocity block is K = (nu/90) (k (x) m + m (x) k), with k and m the 5 x 5
// restrictions of the 1D integer stiffness and mass rows to the window
// (nodes 2i-2 .. 2i+2).  With the generalised eigenvectors k S = m S diag(l),
// S^T m S = I:  K^-1 = (90/nu) (S (x) S) diag(1/(l_a + l_b)) (S (x) S)^T.
// The window is symmetric under reflection, so the eigenvectors split into
// three symmetric and two antisymmetric ones, computed in the reduced bases
// {e0+e4, e1+e3, e2} and {e0-e4, e1-e3}.
// ---------------------------------------------------------------------------
namespace {

// Cyclic Jacobi eigenvalue iteration for a small symmetric matrix a (m x m,
// row-major, destroyed); eigenvalues in w, eigenvectors in the columns of v.
void jacobi_eig(double* a, int m, double* w, double* v) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) v[i * m + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) off += a[p * m + q] * a[p * m + q];
    if (off < 1e-34) break;
    for (int p = 0; p < m; ++p) {
      for (int q = p + 1; q < m; ++q) {
        const double apq = a[p * m + q];
        if (apq == 0.0) continue;
        const double theta = (a[q * m + q] - a[p * m + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {  // columns p, q
          const double akp = a[k * m + p], akq = a[k * m + q];
          a[k * m + p] = c * akp - s * akq;
          a[k * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double apk = a[p * m + k], aqk = a[q * m + k];
          a[p * m + k] = c * apk - s * aqk;
          a[q * m + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double vkp = v[k * m + p], vkq = v[k * m + q];
          v[k * m + p] = c * vkp - s * vkq;
          v[k * m + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  for (int i = 0; i < m; ++i) w[i] = a[i * m + i];
}

// Generalised symmetric eigenproblem A q = l B q, q^T B q = 1 (m <= 5): B = L L^T,
// C = L^-1 A L^-T, C = Q diag(l) Q^T, q = L^-T Q.  Columns of out are the q.
void gen_eig(const double* A, const double* B, int m, double* lam, double* out) {
  double L[25] = {0}, Li[25] = {0}, C[25], T[25], Q[25];
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = B[i * m + j];
      for (int k = 0; k < j; ++k) s -= L[i * m + k] * L[j * m + k];
      L[i * m + j] = (i == j) ? std::sqrt(s) : s / L[j * m + j];
    }
  }
  for (int c = 0; c < m; ++c) {  // Li = L^-1 by forward substitution
    for (int i = 0; i < m; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[i * m + k] * Li[k * m + c];
      Li[i * m + c] = s / L[i * m + i];
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += Li[i * m + k] * A[k * m + j];
      T[i * m + j] = s;
    }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += T[i * m + k] * Li[j * m + k];
      C[i * m + j] = s;
    }
  jacobi_eig(C, m, lam, Q);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += Li[k * m + i] * Q[k * m + j];
      out[i * m + j] = s;
    }
}

}  // namespace

FastDiag interior_fast_diag(double nu) {
  // window offsets -2..2 around an even (vertex) node; k1/m1 rows by parity
  double kw[25], mw[25];
  for (int r = 0; r < 5; ++r)
    for (int c = 0; c < 5; ++c) {
      kw[r * 5 + c] = k1(r & 1, c - r);   // node at offset r-2 has the parity of r
      mw[r * 5 + c] = m1(r & 1, c - r);
    }
  // reduced bases: symmetric {e0+e4, e1+e3, e2}, antisymmetric {e0-e4, e1-e3}
  const double Es[3][5] = {{1, 0, 0, 0, 1}, {0, 1, 0, 1, 0}, {0, 0, 1, 0, 0}};
  const double Eo[2][5] = {{1, 0, 0, 0, -1}, {0, 1, 0, -1, 0}};
  auto project = [&](const double (*E)[5], int m, const double* M, double* out) {
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        double s = 0.0;
        for (int r = 0; r < 5; ++r)
          for (int c = 0; c < 5; ++c) s += E[a][r] * M[r * 5 + c] * E[b][c];
        out[a * m + b] = s;
      }
  };
  double ks[9], ms[9], ko[4], mo[4], ls[3], lo[2], qs[9], qo[4];
  project(Es, 3, kw, ks);
  project(Es, 3, mw, ms);
  project(Eo, 2, kw, ko);
  project(Eo, 2, mw, mo);
  gen_eig(ks, ms, 3, ls, qs);
  gen_eig(ko, mo, 2, lo, qo);
  // Each eigenvector is rescaled so that its entry on the pair {0, 4} (reduced
  // index 0) is 1: S = S' diag(g) with g_k that entry, so
  // K^-1 = (90/nu) (S' (x) S') diag(g_a^2 g_b^2 / (l_a + l_b)) (S' (x) S')^T, and
  // the transforms skip one multiply per coefficient (the kernels take the
  // reduced-index-0 row as 1; every |g_k| is above 0.45 of its column's largest entry).
  FastDiag f;
  double g[5];
  for (int k = 0; k < 3; ++k) g[k] = qs[0 * 3 + k];
  for (int k = 0; k < 2; ++k) g[3 + k] = qo[0 * 2 + k];
  for (int mrow = 0; mrow < 3; ++mrow)
    for (int k = 0; k < 3; ++k) f.se[mrow * 3 + k] = qs[mrow * 3 + k] / g[k];
  for (int mrow = 0; mrow < 2; ++mrow)
    for (int k = 0; k < 2; ++k) f.so[mrow * 2 + k] = qo[mrow * 2 + k] / g[3 + k];
  double lam[5] = {ls[0], ls[1], ls[2], lo[0], lo[1]};
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) f.dinv[a * 5 + b] = (90.0 / nu) * (g[a] * g[a]) * (g[b] * g[b]) / (lam[a] + lam[b]);
  // the fused column operators (see FastDiagT)
  for (int b = 0; b < 5; ++b) {
    for (int m = 0; m < 3; ++m)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += f.se[m * 3 + a] * f.dinv[a * 5 + b] * f.se[j * 3 + a];
        f.gs[b * 9 + m * 3 + j] = s;
      }
    for (int m = 0; m < 2; ++m)
      for (int j = 0; j < 2; ++j) {
        double s = 0.0;
        for (int a = 0; a < 2; ++a) s += f.so[m * 2 + a] * f.dinv[(3 + a) * 5 + b] * f.so[j * 2 + a];
        f.ga[b * 4 + m * 2 + j] = s;
      }
  }
  return f;
}

void edge_fast_diag(double nu, double* tab) {
  double kw[25], mw[25];
  for (int r = 0; r < 5; ++r)
    for (int c = 0; c < 5; ++c) {
      kw[r * 5 + c] = k1(r & 1, c - r);
      mw[r * 5 + c] = m1(r & 1, c - r);
    }
  double lam[5][5];
  int nf[5];
  for (int a = 0; a < 5; ++a) {
    int F[5], m = 0;
    for (int s = 0; s < 5; ++s)
      if (axis_free_mask(a) & (1 << s)) F[m++] = s;
    nf[a] = m;
    double ka[25], ma[25], q[25], l[5];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        ka[i * m + j] = kw[F[i] * 5 + F[j]];
        ma[i * m + j] = mw[F[i] * 5 + F[j]];
      }
    gen_eig(ka, ma, m, l, q);
    double* S = tab + EDGE_S + a * 25;
    for (int k = 0; k < 25; ++k) S[k] = 0.0;
    for (int i = 0; i < m; ++i)
      for (int k = 0; k < m; ++k) S[F[i] * 5 + k] = q[i * m + k];
    for (int k = 0; k < 5; ++k) lam[a][k] = (k < m) ? l[k] : 0.0;
  }
  for (int ay = 0; ay < 5; ++ay)
    for (int ax = 0; ax < 5; ++ax) {
      double* D = tab + EDGE_DINV + (5 * ay + ax) * 25;
      for (int ky = 0; ky < 5; ++ky)
        for (int kx = 0; kx < 5; ++kx)
          D[ky * 5 + kx] = (ky < nf[ay] && kx < nf[ax]) ? (90.0 / nu) / (lam[ay][ky] + lam[ax][kx]) : 0.0;
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

// Dense inverses of the coarsest level's velocity Laplacian block (Dirichlet
// rows identity, 2 (2n+1)^2) and Q1 pressure mass matrix ((n+1)^2), for the
// exact coarse solves of the block-triangular preconditioner.
bool bt_coarse_inverses(int n, double nu, std::vector<double>& GL, std::vector<double>& GM) {
  std::vector<double> A;
  dense_operator(n, nu, A);
  const int nq = 2 * n + 1, np = n + 1;
  const int nL = 2 * nq * nq, N = nL + np * np;
  GL.assign(static_cast<size_t>(nL) * nL, 0.0);
  for (int i = 0; i < nL; ++i)
    for (int j = 0; j < nL; ++j) GL[static_cast<size_t>(i) * nL + j] = A[static_cast<size_t>(i) * N + j];
  const double h = 1.0 / n, c = (h / 6.0) * (h / 6.0);
  auto m = [n](int i, int d) -> double {
    if (d == 0) return (i == 0 || i == n) ? 2.0 : 4.0;
    const int k = i + d;
    return (k < 0 || k > n || (d != 1 && d != -1)) ? 0.0 : 1.0;
  };
  const int nM = np * np;
  GM.assign(static_cast<size_t>(nM) * nM, 0.0);
  for (int j = 0; j < np; ++j)
    for (int i = 0; i < np; ++i)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          const int i2 = i + di, j2 = j + dj;
          if (i2 < 0 || j2 < 0 || i2 > n || j2 > n) continue;
          GM[static_cast<size_t>(j * np + i) * nM + (j2 * np + i2)] = c * m(i, di) * m(j, dj);
        }
  return invert_dense(GL, nL) && invert_dense(GM, nM);
}

}  // namespace sv
