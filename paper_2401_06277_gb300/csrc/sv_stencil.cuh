// sv_stencil.cuh -- matrix-free stencils of the Dirichlet-eliminated Q2-Q1
// Stokes operator on a uniform n x n grid (Section 2.2, Section 2.3).
//
// The global Q2 basis is a tensor product of 1D quadratic Lagrange functions,
// so every block of A is a Kronecker product of assembled 1D matrices:
//   L   = nu (K (x) M + M (x) K)        (K: 1D Q2 stiffness, M: 1D Q2 mass)
//   B_x = -C (x) N,  B_y = -N (x) C     (C_aF = int q_a Psi_F', N_aF = int q_a Psi_F)
// with b(v, p) = -int p div v.  On the rows that survive the elimination of
// the Dirichlet nodes (interior velocity rows, all pressure rows) the 1D rows
// are the interior ones, up to columns that are Dirichlet nodes and therefore
// dropped; so the operator is a translation-invariant stencil (by node parity)
// with a mask.  In integer units:
//   stiffness row  (1/(3h)):  even node [1 -8 14 -8 1],  odd node [-8 16 -8]
//   mass row       (h/30)  :  even node [-1 2 8 2 -1],   odd node [2 16 2]
//   => L coefficients carry the factor nu/90.
//   C column (1/6), Q2 node I against Q1 vertex i:
//        I = 2a   : i = a-1 -> +1,  i = a+1 -> -1
//        I = 2a+1 : i = a   -> +4,  i = a+1 -> -4
//   N column (h/3), Q2 node J against Q1 vertex j:
//        J = 2b   : j = b -> 1;   J = 2b+1 : j = b, b+1 -> 1
//   => B coefficients carry the factor -h/18.
// Only the right-hand side needs the one-sided boundary rows of C and N
// (c1_full / n1_full below).
#pragma once

#ifdef __CUDACC__
#define SV_HD __host__ __device__ __forceinline__ constexpr
#else
#define SV_HD inline constexpr
#endif

namespace sv {

// 1D stiffness row of node F at column F + off, in units of 1/(3h) (interior rows).
SV_HD double k1(int F, int off) {
  if (F & 1) return off == 0 ? 16.0 : ((off == 1 || off == -1) ? -8.0 : 0.0);
  switch (off) {
    case 0: return 14.0;
    case 1: case -1: return -8.0;
    case 2: case -2: return 1.0;
    default: return 0.0;
  }
}

// 1D mass row of node F at column F + off, in units of h/30 (interior rows).
SV_HD double m1(int F, int off) {
  if (F & 1) return off == 0 ? 16.0 : ((off == 1 || off == -1) ? 2.0 : 0.0);
  switch (off) {
    case 0: return 8.0;
    case 1: case -1: return 2.0;
    case 2: case -2: return -1.0;
    default: return 0.0;
  }
}

// C row of a Q1 vertex i at Q2 node 2i + off, in units of 1/6 (interior rows,
// exact on every row once Dirichlet columns are dropped).
SV_HD double crow(int off) {
  switch (off) {
    case -2: return -1.0;
    case -1: return -4.0;
    case 1: return 4.0;
    case 2: return 1.0;
    default: return 0.0;
  }
}

// N row of a Q1 vertex j at Q2 node 2j + off, in units of h/3 (same remark).
SV_HD double nrow(int off) { return (off >= -1 && off <= 1) ? 1.0 : 0.0; }

// Full assembled 1D C entry int q_a Psi_F' (dimensionless), boundary rows included.
SV_HD double c1_full(int a, int F, int n) {
  double v = 0.0;
  if (a >= 1) {  // element a-1, q_a is its local vertex 1; Q2 local nodes 2a-2, 2a-1, 2a
    int l = F - (2 * a - 2);
    if (l == 0) v += -1.0 / 6.0;
    else if (l == 1) v += -2.0 / 3.0;
    else if (l == 2) v += 5.0 / 6.0;
  }
  if (a <= n - 1) {  // element a, q_a is its local vertex 0; Q2 local nodes 2a, 2a+1, 2a+2
    int l = F - 2 * a;
    if (l == 0) v += -5.0 / 6.0;
    else if (l == 1) v += 2.0 / 3.0;
    else if (l == 2) v += 1.0 / 6.0;
  }
  return v;
}

// Full assembled 1D N entry int q_a Psi_F / h, boundary rows included.
SV_HD double n1_full(int a, int F, int n) {
  double v = 0.0;
  if (a >= 1) {
    int l = F - (2 * a - 2);
    if (l == 1) v += 1.0 / 3.0;
    else if (l == 2) v += 1.0 / 6.0;
  }
  if (a <= n - 1) {
    int l = F - 2 * a;
    if (l == 0) v += 1.0 / 6.0;
    else if (l == 1) v += 1.0 / 3.0;
  }
  return v;
}

// Column form of C (units 1/6): coefficient of vertex i in the column of Q2 node I.
SV_HD double ccol(int I, int i) { return crow(I - 2 * i); }
// Column form of N (units h/3).
SV_HD double ncol(int J, int j) { return nrow(J - 2 * j); }

// Per-axis patch class of vertex i (Section 6.3): 0, 1, interior (2), n-1 (3), n (4).
SV_HD int axis_class(int i, int n) {
  return i == 0 ? 0 : (i == 1 ? 1 : (i == n ? 4 : (i == n - 1 ? 3 : 2)));
}

// Number of vertex patches whose 5x5 Q2 window contains Q2 index I on one axis.
SV_HD int axis_mult(int I, int n) {
  int lo = (I - 1) / 2;       // ceil((I-2)/2) for I >= 0
  if (I < 2) lo = 0;
  int hi = (I + 2) / 2;
  if (hi > n) hi = n;
  return hi - lo + 1;
}

}  // namespace sv
