"""Plain FP64 CPU oracle for Q2-Q1 Stokes with additive-Vanka multigrid and FGMRES.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct reference
the CUDA library is checked against.  Only the test-suite, the smoke check and
the benchmark's CPU-baseline leg may import it; the library never calls it.
It shares no code with the CUDA path (its inputs come from ``stokes_inputs``,
which holds problem data only).

What it follows (paper: Spies, Olson, MacLachlan, "Exploiting mesh structure to
improve multigrid performance for saddle point problems"):
  * Section 2.1: -nu Lap u + grad p = f, div u = 0 on the unit square, with the
    weak forms a(u, v) = nu int grad u : grad v and b(v, p) (sign: see below).
  * Section 2.2: Q2-Q1 Taylor-Hood on a uniform quadrilateral grid;
    L_ij = a(psi_j, psi_i), B_kj = b(psi_j, phi_k), A = [[L, B^T], [B, 0]].
  * Section 3, Algorithm 1 (MG): V-cycle, FE interpolation P, restriction P^T,
    exact solve on the coarsest level 0.
  * Section 3.2, Algorithm 3 (additive Vanka): vertex patches of 2x2
    elements, A_i = V_i A V_i^T solved exactly, x += sum_i V_i^T W_i delta_i.
  * Section 6.3: on a uniform grid there are 25 distinct patch matrices.
  * Section 2.2 / 6.8: FGMRES, right-preconditioned by the V-cycle.

Readings where the paper is silent (each is listed in the design notes):
  * Dirichlet velocity on every edge, eliminated symmetrically (identity rows
    and columns, lifting moved to the right-hand side).
  * b(v, p) = -int p div v (the sign that integrating grad p . v by parts
    gives for the strong form -nu Lap u + grad p = f); the printed "+" sign
    only flips the sign of the discrete pressure (A -> D A D, D = diag(I, -I)).
  * W_i = omega * diag(1 / m_j), m_j = number of patches holding dof j.
  * Patch dof order: u_x 5x5 window (row-major), u_y window, then p.
  * Pressure is defined up to a constant: the coarse solve and the direct
    reference solve use the bordered system [[A, e], [e^T, 0]], e = (0, M_p 1).
  * FGMRES(m): modified Gram-Schmidt Arnoldi, Givens rotations, stop when the
    estimated residual norm drops below rtol * ||b - A x0||.

Parity is pinned by the tests in tests/test_oracle_*.py (closed-form element
matrices, symmetry, polynomial exactness, O(h^3)/O(h^2) convergence, Galerkin
identity, patch-class counts, brute-force patch solves, LU references).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ----------------------------------------------------------------------------
# Reference elements (Section 2.2): 1D quadratic and linear Lagrange bases on
# [0, 1] with nodes {0, 1/2, 1} and {0, 1}; 2D bases are tensor products.
# ----------------------------------------------------------------------------


def gauss_legendre_01(k: int) -> tuple[np.ndarray, np.ndarray]:
    """k-point Gauss-Legendre rule on [0, 1] (exact for degree 2k-1)."""
    t, w = np.polynomial.legendre.leggauss(k)
    return 0.5 * (t + 1.0), 0.5 * w


def q2_1d(t: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Values and d/dt of the three 1D quadratic Lagrange functions (nodes 0, 1/2, 1)."""
    t = np.asarray(t, dtype=np.float64)
    v = np.stack([(1 - t) * (1 - 2 * t), 4 * t * (1 - t), t * (2 * t - 1)])
    d = np.stack([4 * t - 3, 4 - 8 * t, 4 * t - 1])
    return v, d


def q1_1d(t: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Values and d/dt of the two 1D linear Lagrange functions (nodes 0, 1)."""
    t = np.asarray(t, dtype=np.float64)
    v = np.stack([1 - t, t])
    d = np.stack([-np.ones_like(t), np.ones_like(t)])
    return v, d


def q2_basis_2d(s: np.ndarray, t: np.ndarray):
    """Q2 element basis at points (s, t): values, d/ds, d/dt; local node (a, b) -> b*3 + a."""
    vs, ds = q2_1d(s)
    vt, dt = q2_1d(t)
    val = np.einsum("bq,aq->baq", vt, vs).reshape(9, -1)
    dds = np.einsum("bq,aq->baq", vt, ds).reshape(9, -1)
    ddt = np.einsum("bq,aq->baq", dt, vs).reshape(9, -1)
    return val, dds, ddt


def q1_basis_2d(s: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Q1 element basis values at points (s, t); local vertex (a, b) -> b*2 + a."""
    vs, _ = q1_1d(s)
    vt, _ = q1_1d(t)
    return np.einsum("bq,aq->baq", vt, vs).reshape(4, -1)


def element_matrices(h: float) -> dict[str, np.ndarray]:
    """Element matrices on an h x h square by 3x3 Gauss quadrature (exact here).

    stiff[i, j] = int grad psi_i . grad psi_j     (9 x 9, scalar Q2)
    mass[i, j]  = int psi_i psi_j                  (9 x 9)
    bx[k, j]    = -int phi_k d(psi_j)/dx           (4 x 9)
    by[k, j]    = -int phi_k d(psi_j)/dy           (4 x 9)
    pmass[k, l] = int phi_k phi_l                  (4 x 4, Q1)
    """
    g, w = gauss_legendre_01(3)
    s = np.tile(g, 3)                                 # s fastest
    t = np.repeat(g, 3)
    wq = np.repeat(w, 3) * np.tile(w, 3) * h * h
    val, dds, ddt = q2_basis_2d(s, t)
    dx, dy = dds / h, ddt / h
    phi = q1_basis_2d(s, t)
    stiff = (dx * wq) @ dx.T + (dy * wq) @ dy.T
    mass = (val * wq) @ val.T
    # the exact matrices are symmetric; averaging with the transpose removes the
    # rounding-order asymmetry of the quadrature sums, so A is symmetric bit for bit
    return {
        "stiff": 0.5 * (stiff + stiff.T),
        "mass": 0.5 * (mass + mass.T),
        "bx": -((phi * wq) @ dx.T),
        "by": -((phi * wq) @ dy.T),
        "pmass": (phi * wq) @ phi.T,
    }


# ----------------------------------------------------------------------------
# Global numbering (Section 2.3, lexicographic): u_x, u_y on the (2n+1)^2 Q2
# nodes, then p on the (n+1)^2 vertices; x index fastest.
# ----------------------------------------------------------------------------


@dataclass
class Mesh:
    n: int

    @property
    def h(self) -> float:
        return 1.0 / self.n

    @property
    def nq(self) -> int:
        return 2 * self.n + 1

    @property
    def np_(self) -> int:
        return self.n + 1

    @property
    def nvel(self) -> int:
        return self.nq * self.nq

    @property
    def ndof(self) -> int:
        return 2 * self.nvel + self.np_ * self.np_

    def ux(self, I, J):
        return np.asarray(J) * self.nq + np.asarray(I)

    def uy(self, I, J):
        return self.nvel + np.asarray(J) * self.nq + np.asarray(I)

    def p(self, i, j):
        return 2 * self.nvel + np.asarray(j) * self.np_ + np.asarray(i)

    def dirichlet_mask(self) -> np.ndarray:
        """True on velocity dofs of boundary Q2 nodes (both components)."""
        m = np.zeros(self.ndof, dtype=bool)
        k = np.arange(self.nq)
        on = (k == 0) | (k == self.nq - 1)
        bd = (on[None, :] | on[:, None]).ravel()       # [J, I] flattened
        m[: self.nvel] = bd
        m[self.nvel: 2 * self.nvel] = bd
        return m


def assemble_blocks(mesh: Mesh):
    """Assemble scalar Q2 stiffness, Q2 mass, B_x, B_y and Q1 mass (CSR) element by element."""
    n, nq, npn = mesh.n, mesh.nq, mesh.np_
    em = element_matrices(mesh.h)
    ex, ey = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    ex, ey = ex.ravel(), ey.ravel()
    # local Q2 node (a, b) of element (ex, ey) is global node (2ex + a, 2ey + b)
    q2 = np.stack([(2 * ey + b) * nq + (2 * ex + a) for b in range(3) for a in range(3)])
    q1 = np.stack([(ey + b) * npn + (ex + a) for b in range(2) for a in range(2)])

    def asm(local, rows, cols, shape):
        r = np.repeat(rows[:, None, :], cols.shape[0], axis=1)
        c = np.repeat(cols[None, :, :], rows.shape[0], axis=0)
        v = np.broadcast_to(local[:, :, None], r.shape)
        return sp.coo_matrix((v.ravel(), (r.ravel(), c.ravel())), shape=shape).tocsr()

    K = asm(em["stiff"], q2, q2, (nq * nq, nq * nq))
    M = asm(em["mass"], q2, q2, (nq * nq, nq * nq))
    Bx = asm(em["bx"], q1, q2, (npn * npn, nq * nq))
    By = asm(em["by"], q1, q2, (npn * npn, nq * nq))
    Mp = asm(em["pmass"], q1, q1, (npn * npn, npn * npn))
    return K, M, Bx, By, Mp


@dataclass
class Level:
    """One grid level: the eliminated operator and everything Vanka needs."""

    mesh: Mesh
    nu: float
    A: sp.csr_matrix = None          # Dirichlet-eliminated, symmetric
    A_full: sp.csr_matrix = None     # before elimination
    Mu: sp.csr_matrix = None         # scalar Q2 mass
    Mp: sp.csr_matrix = None         # Q1 mass
    dmask: np.ndarray = None
    patch_dofs: np.ndarray = None    # [(n+1)^2, 51], -1 where the window leaves the domain
    patch_class: np.ndarray = None   # [(n+1)^2]
    class_inv: dict = field(default_factory=dict)   # class -> (slots, inverse)
    mult: np.ndarray = None          # m_j, patches holding dof j
    P: sp.csr_matrix = None          # prolongation from the next coarser level


def stokes_operator(mesh: Mesh, nu: float):
    """A_full = [[nu K, 0, Bx^T], [0, nu K, By^T], [Bx, By, 0]] and its symmetric elimination."""
    K, M, Bx, By, Mp = assemble_blocks(mesh)
    Z = sp.csr_matrix((mesh.nvel, mesh.nvel))
    Zp = sp.csr_matrix((mesh.np_ ** 2, mesh.np_ ** 2))
    A_full = sp.bmat([[nu * K, Z, Bx.T], [Z, nu * K, By.T], [Bx, By, Zp]], format="csr")
    d = mesh.dirichlet_mask()
    keep = sp.diags((~d).astype(np.float64))
    A = (keep @ A_full @ keep + sp.diags(d.astype(np.float64))).tocsr()
    A.eliminate_zeros()
    return A, A_full, M, Mp, d


def assemble_rhs(level: Level, f_nodal: np.ndarray, u_dir: np.ndarray) -> np.ndarray:
    """b = [M f on free velocity rows - lifting ; -B_D u_D ; u_D on Dirichlet rows].

    f_nodal and u_dir are [2, 2n+1, 2n+1]; only boundary entries of u_dir are read.
    """
    mesh = level.mesh
    nv = mesh.nvel
    F = np.zeros(mesh.ndof)
    F[:nv] = level.Mu @ f_nodal[0].ravel()
    F[nv: 2 * nv] = level.Mu @ f_nodal[1].ravel()
    g = np.zeros(mesh.ndof)
    d = level.dmask
    g[:2 * nv] = np.concatenate([u_dir[0].ravel(), u_dir[1].ravel()])
    g[~d] = 0.0
    b = F - level.A_full @ g
    b[d] = g[d]
    return b


# ----------------------------------------------------------------------------
# Vanka patches (Section 3.2, Section 6.3)
# ----------------------------------------------------------------------------

NSLOT = 51


def patch_slots(mesh: Mesh, i: int, j: int) -> np.ndarray:
    """Global dofs of the vertex patch at (i, j) in slot order, -1 outside the domain.

    Slots 0..24: u_x on Q2 nodes (2i+dI, 2j+dJ), dI, dJ in -2..2, slot (dJ+2)*5 + (dI+2);
    slots 25..49: u_y on the same nodes; slot 50: p at vertex (i, j)."""
    out = -np.ones(NSLOT, dtype=np.int64)
    for dJ in range(-2, 3):
        for dI in range(-2, 3):
            I, J = 2 * i + dI, 2 * j + dJ
            if 0 <= I < mesh.nq and 0 <= J < mesh.nq:
                s = (dJ + 2) * 5 + (dI + 2)
                out[s] = mesh.ux(I, J)
                out[25 + s] = mesh.uy(I, J)
    out[50] = mesh.p(i, j)
    return out


def patch_table(mesh: Mesh) -> np.ndarray:
    """patch_slots for every vertex at once: [(n+1)^2, 51], vertex (i, j) at row j*(n+1) + i."""
    n, nq = mesh.n, mesh.nq
    i = np.arange(n + 1)
    d = np.arange(-2, 3)
    I = 2 * i[:, None] + d[None, :]                        # [i, dI]
    okI = (I >= 0) & (I < nq)
    # [j, i, dJ, dI]
    J = I
    g = J[:, None, :, None] * nq + I[None, :, None, :]
    ok = okI[:, None, :, None] & okI[None, :, None, :]
    nv = (n + 1) ** 2
    win = np.where(ok, g, -1).reshape(nv, 25)
    out = np.empty((nv, NSLOT), dtype=np.int64)
    out[:, :25] = win
    out[:, 25:50] = np.where(win >= 0, win + mesh.nvel, -1)
    out[:, 50] = 2 * mesh.nvel + np.arange(nv)
    return out


def axis_class(i: int, n: int) -> int:
    """Per-axis patch class of vertex index i: 0, 1, interior (2), n-1 (3), n (4)."""
    if i == 0:
        return 0
    if i == 1:
        return 1
    if i == n:
        return 4
    if i == n - 1:
        return 3
    return 2


def build_patches(level: Level, per_patch: bool = False) -> None:
    """Patch index table, classes, multiplicities and patch inverses.

    per_patch=False ("tuned" Vanka, Section 6.3): one inverse per class, taken
    from the first patch of the class; tests check that every patch of a class
    has a bitwise-equal A_i.  per_patch=True ("simple" Vanka): every patch gets
    its own inverse.
    """
    mesh = level.mesh
    n = mesh.n
    nv = (n + 1) ** 2
    dofs = patch_table(mesh)
    ac = np.array([axis_class(i, n) for i in range(n + 1)])
    cls = (5 * ac[:, None] + ac[None, :]).ravel()          # [j, i] -> 5 cls(j) + cls(i)
    level.patch_dofs, level.patch_class = dofs, cls
    level.mult = np.bincount(dofs[dofs >= 0], minlength=mesh.ndof).astype(np.float64)
    A = level.A
    level.class_inv = {}
    if per_patch:
        level.class_inv["per_patch"] = [_patch_inverse(A, dofs[k]) for k in range(nv)]
        return
    for c in np.unique(cls):
        first = int(np.flatnonzero(cls == c)[0])
        level.class_inv[int(c)] = _patch_inverse(A, dofs[first])


def patch_matrix(A: sp.csr_matrix, dofs: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """A_i = V_i A V_i^T on the in-domain slots of a patch (dense)."""
    slots = np.flatnonzero(dofs >= 0)
    g = dofs[slots]
    return slots, A[g][:, g].toarray()


def _patch_inverse(A: sp.csr_matrix, dofs: np.ndarray):
    slots, Ai = patch_matrix(A, dofs)
    lu = sla.lu_factor(Ai)                      # dense LU with partial pivoting
    inv = sla.lu_solve(lu, np.eye(len(slots)))
    return slots, inv


def vanka_correction(level: Level, r: np.ndarray) -> np.ndarray:
    """sum_i V_i^T A_i^{-1} V_i r, every patch using the same residual r (Algorithm 3)."""
    dofs, cls = level.patch_dofs, level.patch_class
    acc = np.zeros_like(r)
    if "per_patch" in level.class_inv:
        for k, (slots, inv) in enumerate(level.class_inv["per_patch"]):
            g = dofs[k, slots]
            np.add.at(acc, g, inv @ r[g])
        return acc
    for c, (slots, inv) in level.class_inv.items():
        sel = np.flatnonzero(cls == c)
        g = dofs[sel][:, slots]                  # [patches, size]
        delta = r[g] @ inv.T                      # delta_i = A_c^{-1} r_i
        acc += np.bincount(g.ravel(), weights=delta.ravel(), minlength=len(r))
    return acc


def vanka_sweep(level: Level, x: np.ndarray, b: np.ndarray, omega: float,
                weights: str = "multiplicity") -> np.ndarray:
    """One additive Vanka sweep: x + sum_i V_i^T W_i A_i^{-1} V_i (b - A x).

    weights="multiplicity": W_i = omega diag(1/m_j); weights="identity": W_i = omega I."""
    r = b - level.A @ x
    c = vanka_correction(level, r)
    if weights == "multiplicity":
        return x + omega * c / level.mult
    return x + omega * c


# ----------------------------------------------------------------------------
# Grid transfer (Section 3): FE interpolation P and restriction P^T
# ----------------------------------------------------------------------------


def interp_1d_q2(nc: int) -> np.ndarray:
    """Values of the coarse 1D Q2 basis (nc elements) at the fine Q2 nodes (2nc elements)."""
    nf = 2 * nc
    P = np.zeros((2 * nf + 1, 2 * nc + 1))
    for F in range(2 * nf + 1):
        x = F / (2 * nf)
        e = min(int(np.floor(x * nc)), nc - 1)
        t = x * nc - e
        v, _ = q2_1d(np.array([t]))
        for a in range(3):
            P[F, 2 * e + a] += v[a, 0]
    return P


def interp_1d_q1(nc: int) -> np.ndarray:
    """Values of the coarse 1D Q1 basis at the fine vertices."""
    nf = 2 * nc
    P = np.zeros((nf + 1, nc + 1))
    for F in range(nf + 1):
        x = F / nf
        e = min(int(np.floor(x * nc)), nc - 1)
        t = x * nc - e
        v, _ = q1_1d(np.array([t]))
        for a in range(2):
            P[F, e + a] += v[a, 0]
    return P


def prolongation(fine: Mesh, coarse: Mesh) -> sp.csr_matrix:
    """Block-diagonal FE interpolation, zero on fine Dirichlet rows and coarse Dirichlet columns."""
    assert fine.n == 2 * coarse.n
    p2 = interp_1d_q2(coarse.n)
    p1 = interp_1d_q1(coarse.n)
    Pq = sp.kron(sp.csr_matrix(p2), sp.csr_matrix(p2))
    Pp = sp.kron(sp.csr_matrix(p1), sp.csr_matrix(p1))
    P = sp.block_diag([Pq, Pq, Pp], format="csr")
    df = (~fine.dirichlet_mask()).astype(np.float64)
    dc = (~coarse.dirichlet_mask()).astype(np.float64)
    P = (sp.diags(df) @ P @ sp.diags(dc)).tocsr()
    P.eliminate_zeros()
    return P


# ----------------------------------------------------------------------------
# Braess-Sarazin relaxation (Section 3.1, Algorithm 2: the inexact variant)
# ----------------------------------------------------------------------------


@dataclass
class BSParams:
    """t scales D = diag(L); omega is omega_BS; the Schur system is relaxed by
    `jacobi_iters` weighted-Jacobi steps of weight `jacobi_weight` from zero
    (the paper leaves all four to experiment; the defaults are the best of a
    search over t in {1, 1.25, 1.5, 2, 2.5}, omega in {0.8, 1}, weight in
    {0.7, 1}, iterations in {1, 2, 3}: fewest FGMRES(30) iterations to 1e-8 with
    V(2,2) at 32^2 and 64^2)."""
    t: float = 1.0
    omega: float = 1.0
    jacobi_weight: float = 1.0
    jacobi_iters: int = 2


def bs_blocks(level: Level):
    """L (velocity block of the eliminated A: identity on Dirichlet rows), B (pressure rows), D = diag(L)."""
    nv2 = 2 * level.mesh.nvel
    A = level.A.tocsr()
    L = A[:nv2, :nv2]
    B = A[nv2:, :nv2]
    return L, B, L.diagonal()


def bs_schur(level: Level, t: float) -> sp.csr_matrix:
    """S = -(1/t) B D^-1 B^T, the Schur complement of [[tD, B^T], [B, 0]]."""
    _, B, D = bs_blocks(level)
    return (-(1.0 / t) * (B @ sp.diags(1.0 / D) @ B.T)).tocsr()


def braess_sarazin_sweep(level: Level, x: np.ndarray, b: np.ndarray, prm: BSParams,
                         schur: str = "jacobi") -> np.ndarray:
    """One Braess-Sarazin step (Algorithm 2), D = diag(L), S = -(1/t) B D^-1 B^T:
      1. approximately solve S dp = r_p - (1/t) B D^-1 r_u (weighted Jacobi from 0, or
         schur="exact": the minimum-norm solution; S is singular in the pressure constant),
      2. du = (1/t) D^-1 (r_u - B^T dp)   (Eq. bseq2),
      3. p += omega_BS dp, u += omega_BS du."""
    nv2 = 2 * level.mesh.nvel
    _, B, D = bs_blocks(level)
    r = b - level.A @ x
    ru, rp = r[:nv2], r[nv2:]
    t = prm.t
    g = rp - (1.0 / t) * (B @ (ru / D))
    S = bs_schur(level, t)
    if schur == "exact":
        dp = np.linalg.lstsq(S.toarray(), g, rcond=None)[0]
    else:
        dS = S.diagonal()
        dp = np.zeros_like(g)
        for _ in range(prm.jacobi_iters):
            dp = dp + prm.jacobi_weight * (g - S @ dp) / dS
    du = (1.0 / t) * (ru - B.T @ dp) / D
    return x + prm.omega * np.concatenate([du, dp])


def schur_uzawa_sweep(level: Level, x: np.ndarray, b: np.ndarray, prm: BSParams,
                      schur: str = "jacobi") -> np.ndarray:
    """One Schur-Uzawa step (Section 3.3, Algorithm 4), the block lower-triangular
    approximation [[tD, 0], [B, S]] [du; dp] = [r_u; r_p] with S = -(1/t) B D^-1 B^T:
      1. du = (1/t) D^-1 r_u,
      2. approximately solve S dp = r_p - B du (weighted Jacobi from 0, or the
         minimum-norm exact solve),
      3. u += omega du, p += omega dp (the paper's algorithm is undamped: omega = 1).
    The paper's prose writes the Schur equation as S dp = B du - r_p; with its
    S = -(1/t) B D^-1 B^T that contradicts the block system it is derived from, which
    is followed here."""
    nv2 = 2 * level.mesh.nvel
    _, B, D = bs_blocks(level)
    r = b - level.A @ x
    ru, rp = r[:nv2], r[nv2:]
    du = (1.0 / prm.t) * ru / D
    g = rp - B @ du
    S = bs_schur(level, prm.t)
    if schur == "exact":
        dp = np.linalg.lstsq(S.toarray(), g, rcond=None)[0]
    else:
        dS = S.diagonal()
        dp = np.zeros_like(g)
        for _ in range(prm.jacobi_iters):
            dp = dp + prm.jacobi_weight * (g - S @ dp) / dS
    return x + prm.omega * np.concatenate([du, dp])


# ----------------------------------------------------------------------------
# Hierarchy, coarse solve, V-cycle (Algorithm 1)
# ----------------------------------------------------------------------------


@dataclass
class Hierarchy:
    levels: list            # levels[0] = coarsest
    nu: float
    omega: float
    nu1: int
    nu2: int
    coarse_lu: tuple = None
    weights: str = "multiplicity"
    smoother: str = "vanka"          # or "bs" (Braess-Sarazin, Algorithm 2), "su" (Schur-Uzawa, Algorithm 4)
    bs: BSParams = None
    gamma: int = 1                   # coarse-grid cycles per level: 1 = V-cycle, 2 = W-cycle


def build_level(n: int, nu: float, per_patch: bool = False) -> Level:
    mesh = Mesh(n)
    A, A_full, Mu, Mp, d = stokes_operator(mesh, nu)
    lv = Level(mesh=mesh, nu=nu, A=A, A_full=A_full, Mu=Mu, Mp=Mp, dmask=d)
    build_patches(lv, per_patch=per_patch)
    return lv


def bordered_matrix(level: Level) -> sp.csr_matrix:
    """[[A, e], [e^T, 0]] with e = (0, M_p 1): fixes the pressure constant (int p = 0)."""
    mesh = level.mesh
    e = np.zeros(mesh.ndof)
    e[2 * mesh.nvel:] = level.Mp @ np.ones(mesh.np_ ** 2)
    return sp.bmat([[level.A, sp.csr_matrix(e[:, None])],
                    [sp.csr_matrix(e[None, :]), None]], format="csc")


def build_hierarchy(n: int, nu: float = 1.0, coarse_n: int = 4, omega: float = 0.7,
                    nu1: int = 2, nu2: int = 2, per_patch: bool = False,
                    weights: str = "multiplicity", smoother: str = "vanka",
                    bs: BSParams | None = None, gamma: int = 1) -> Hierarchy:
    """Rediscretised levels n, n/2, ..., coarse_n (Section 3: geometric multigrid)."""
    sizes = []
    m = n
    while m > coarse_n:
        sizes.append(m)
        assert m % 2 == 0, "n must be coarse_n * 2^k"
        m //= 2
    assert m == coarse_n, "n must be coarse_n * 2^k"
    sizes.append(coarse_n)
    levels = [build_level(s, nu, per_patch) for s in reversed(sizes)]
    for l in range(1, len(levels)):
        levels[l].P = prolongation(levels[l].mesh, levels[l - 1].mesh)
    H = Hierarchy(levels=levels, nu=nu, omega=omega, nu1=nu1, nu2=nu2, weights=weights,
                  smoother=smoother, bs=bs if bs is not None else BSParams(), gamma=gamma)
    Kb = bordered_matrix(levels[0]).toarray()
    H.coarse_lu = sla.lu_factor(Kb)
    return H


def coarse_solve(H: Hierarchy, r: np.ndarray) -> np.ndarray:
    """e_0 = A_0^{-1} r_0 through the bordered system (exact, dense LU)."""
    rr = np.concatenate([r, [0.0]])
    return sla.lu_solve(H.coarse_lu, rr)[:-1]


def vcycle(H: Hierarchy, b: np.ndarray, l: int | None = None) -> np.ndarray:
    """Algorithm 1 with a zero initial guess: nu1 sweeps, restrict, recurse, correct, nu2 sweeps.
    With H.gamma = 2 the coarse problem A_c e = r_c is iterated twice (W-cycle): the second
    cycle starts from the first's result, e += cycle(r_c - A_c e)."""
    if l is None:
        l = len(H.levels) - 1
    if l == 0:
        return coarse_solve(H, b)
    lv = H.levels[l]
    x = np.zeros_like(b)
    for _ in range(H.nu1):
        x = relax(H, lv, x, b)
    r = b - lv.A @ x
    rc = lv.P.T @ r
    if l == 1:
        ec = coarse_solve(H, rc)
    else:
        ec = vcycle(H, rc, l - 1)
        Ac = H.levels[l - 1].A
        for _ in range(H.gamma - 1):
            ec = ec + vcycle(H, rc - Ac @ ec, l - 1)
    x = x + lv.P @ ec
    for _ in range(H.nu2):
        x = relax(H, lv, x, b)
    return x


def relax(H: Hierarchy, lv: Level, x: np.ndarray, b: np.ndarray) -> np.ndarray:
    """One sweep of the hierarchy's relaxation: additive Vanka (Algorithm 3), Braess-Sarazin
    (Algorithm 2) or Schur-Uzawa (Algorithm 4)."""
    if H.smoother == "bs":
        return braess_sarazin_sweep(lv, x, b, H.bs)
    if H.smoother == "su":
        return schur_uzawa_sweep(lv, x, b, H.bs)
    return vanka_sweep(lv, x, b, H.omega, H.weights)


# ----------------------------------------------------------------------------
# Block-triangular preconditioner (Section 3.4, Algorithm 5)
# ----------------------------------------------------------------------------


@dataclass
class BTParams:
    """Section 6.8's settings: 3 V(3,3) cycles per block, weighted Jacobi of weight
    0.6 on the pressure mass matrix and 1.0 on the velocity Laplacian."""
    cycles: int = 3
    nu1: int = 3
    nu2: int = 3
    omega_p: float = 0.6
    omega_u: float = 1.0


def scalar_vcycle(mats: list, prols: list, b: np.ndarray, l: int, omega: float, nu1: int, nu2: int,
                  coarse_inv: np.ndarray, x0: np.ndarray | None = None) -> np.ndarray:
    """One V(nu1, nu2) cycle of multigrid on the SPD matrices mats[l] (level 0 coarsest),
    weighted-Jacobi smoothing, prolongations prols[l] (level l-1 -> l), exact coarse solve."""
    if l == 0:
        return coarse_inv @ b
    A = mats[l]
    dinv = 1.0 / A.diagonal()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    for _ in range(nu1):
        x = x + omega * dinv * (b - A @ x)
    P = prols[l]
    x = x + P @ scalar_vcycle(mats, prols, P.T @ (b - A @ x), l - 1, omega, nu1, nu2, coarse_inv)
    for _ in range(nu2):
        x = x + omega * dinv * (b - A @ x)
    return x


def block_triangular_setup(H: Hierarchy) -> dict:
    """Per level: the velocity Laplacian block L (eliminated: identity on Dirichlet rows),
    the pressure mass matrix M, B, and the blocks of the prolongation."""
    out = {"L": [], "M": [], "B": [], "PL": [None], "PM": [None]}
    for l, lv in enumerate(H.levels):
        nv2 = 2 * lv.mesh.nvel
        A = lv.A.tocsr()
        out["L"].append(A[:nv2, :nv2].tocsr())
        out["B"].append(A[nv2:, :nv2].tocsr())
        out["M"].append(lv.Mp.tocsr())
        if l > 0:
            P = lv.P.tocsr()
            out["PL"].append(P[:nv2, :2 * H.levels[l - 1].mesh.nvel].tocsr())
            out["PM"].append(P[nv2:, 2 * H.levels[l - 1].mesh.nvel:].tocsr())
    out["Linv0"] = np.linalg.inv(out["L"][0].toarray())
    out["Minv0"] = np.linalg.inv(out["M"][0].toarray())
    return out


def block_triangular_apply(H: Hierarchy, bt: dict, r: np.ndarray, prm: BTParams = BTParams(),
                           exact: bool = False) -> np.ndarray:
    """Algorithm 5: approximately solve M dp = -r_p, then L du = r_u - B^T dp, each by
    `cycles` multigrid V(nu1, nu2) cycles (iterative refinement from zero), or exactly."""
    top = len(H.levels) - 1
    nv2 = 2 * H.levels[top].mesh.nvel
    ru, rp = r[:nv2], r[nv2:]
    M, L, B = bt["M"][top], bt["L"][top], bt["B"][top]

    def solve(mats, prols, rhs, omega, cinv):
        if exact:
            return spla.spsolve(mats[top].tocsc(), rhs)
        x = np.zeros_like(rhs)
        for _ in range(prm.cycles):
            x = x + scalar_vcycle(mats, prols, rhs - mats[top] @ x, top, omega, prm.nu1, prm.nu2, cinv)
        return x

    dp = solve(bt["M"], bt["PM"], -rp, prm.omega_p, bt["Minv0"])
    du = solve(bt["L"], bt["PL"], ru - B.T @ dp, prm.omega_u, bt["Linv0"])
    return np.concatenate([du, dp])


# ----------------------------------------------------------------------------
# FGMRES(m), right-preconditioned (Saad's flexible GMRES)
# ----------------------------------------------------------------------------


@dataclass
class FGMRESResult:
    x: np.ndarray
    iters: int
    relres: float           # true ||b - A x|| / ||b - A x0|| at exit
    converged: bool
    history: list


def fgmres(A, b: np.ndarray, x0: np.ndarray, precond, restart: int = 30,
           rtol: float = 1e-8, maxit: int = 1000) -> FGMRESResult:
    x = x0.copy()
    r = b - A @ x
    beta0 = np.linalg.norm(r)
    hist = [1.0]
    if beta0 == 0.0:
        return FGMRESResult(x, 0, 0.0, True, hist)
    it = 0
    while it < maxit:
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((m + 1, len(b)))
        Z = np.zeros((m, len(b)))
        Hm = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = A @ Z[j]
            for i in range(j + 1):                      # modified Gram-Schmidt
                Hm[i, j] = w @ V[i]
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] != 0.0:
                V[j + 1] = w / Hm[j + 1, j]
            for i in range(j):                           # previous rotations
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            d = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = Hm[j, j] / d, Hm[j + 1, j] / d
            Hm[j, j] = d
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / beta0)
            if abs(g[j + 1]) <= rtol * beta0 or it >= maxit:
                break
        y = sla.solve_triangular(Hm[:k, :k], g[:k])
        x = x + Z[:k].T @ y
        r = b - A @ x
        if np.linalg.norm(r) <= rtol * beta0:
            break
    rel = np.linalg.norm(b - A @ x) / beta0
    return FGMRESResult(x, it, rel, rel <= rtol, hist)


def initial_guess(level: Level, b: np.ndarray) -> np.ndarray:
    """x0: zero on free rows, the Dirichlet data on Dirichlet rows."""
    x0 = np.zeros_like(b)
    x0[level.dmask] = b[level.dmask]
    return x0


def solve(H: Hierarchy, b: np.ndarray, restart: int = 30, rtol: float = 1e-8,
          maxit: int = 1000, x0: np.ndarray | None = None) -> FGMRESResult:
    fine = H.levels[-1]
    if x0 is None:
        x0 = initial_guess(fine, b)
    return fgmres(fine.A, b, x0, lambda v: vcycle(H, v), restart, rtol, maxit)


# ----------------------------------------------------------------------------
# Direct reference solve, pressure normalisation, errors, adjoint
# ----------------------------------------------------------------------------


def direct_solve(level: Level, b: np.ndarray) -> np.ndarray:
    """Exact discrete solution with int p = 0 (sparse LU of the bordered system)."""
    K = bordered_matrix(level)
    return spla.spsolve(K, np.concatenate([b, [0.0]]))[:-1]


def normalize_pressure(level: Level, x: np.ndarray) -> np.ndarray:
    """Shift p so that int p_h = 0 (Q1-mass weighted mean)."""
    mesh = level.mesh
    y = x.copy()
    p = y[2 * mesh.nvel:]
    ones = np.ones_like(p)
    y[2 * mesh.nvel:] = p - (ones @ (level.Mp @ p)) / (ones @ (level.Mp @ ones))
    return y


def l2_errors(level: Level, x: np.ndarray, u_exact, p_exact, nq_gauss: int = 4):
    """||u - u_h||_L2 and ||p - p_h||_L2 by nq_gauss^2 Gauss points per element."""
    mesh = level.mesh
    n, h, nq, npn = mesh.n, mesh.h, mesh.nq, mesh.np_
    g, w = gauss_legendre_01(nq_gauss)
    s = np.tile(g, nq_gauss)
    t = np.repeat(g, nq_gauss)
    wq = np.tile(w, nq_gauss) * np.repeat(w, nq_gauss) * h * h
    val, _, _ = q2_basis_2d(s, t)
    phi = q1_basis_2d(s, t)
    ux = x[: mesh.nvel].reshape(nq, nq)
    uy = x[mesh.nvel: 2 * mesh.nvel].reshape(nq, nq)
    pp = x[2 * mesh.nvel:].reshape(npn, npn)
    eu2 = ep2 = 0.0
    for ey in range(n):
        for ex in range(n):
            lx = ux[2 * ey: 2 * ey + 3, 2 * ex: 2 * ex + 3].ravel()
            ly = uy[2 * ey: 2 * ey + 3, 2 * ex: 2 * ex + 3].ravel()
            lp = pp[ey: ey + 2, ex: ex + 2].ravel()
            X = (ex + s) * h
            Y = (ey + t) * h
            ue = u_exact(X, Y)
            eu2 += wq @ ((lx @ val - ue[0]) ** 2 + (ly @ val - ue[1]) ** 2)
            ep2 += wq @ ((lp @ phi - p_exact(X, Y)) ** 2)
    return np.sqrt(eu2), np.sqrt(ep2)


def rhs_map(level: Level) -> sp.csr_matrix:
    """The linear map f_nodal (2 (2n+1)^2) -> its part of b: M f on free velocity rows, 0 elsewhere."""
    mesh = level.mesh
    Mb = sp.block_diag([level.Mu, level.Mu], format="csr")
    free = (~level.dmask[: 2 * mesh.nvel]).astype(np.float64)
    Mt = sp.diags(free) @ Mb
    pad = sp.csr_matrix((mesh.np_ ** 2, 2 * mesh.nvel))
    return sp.vstack([Mt, pad], format="csr")


def misfit(level: Level, x: np.ndarray, u_target: np.ndarray) -> float:
    """J = 1/2 ||u - u_target||_2^2 over all velocity nodal values."""
    nv2 = 2 * level.mesh.nvel
    d = x[:nv2] - u_target.ravel()
    return 0.5 * float(d @ d)


def adjoint_gradient_dense(level: Level, f_nodal: np.ndarray, u_dir: np.ndarray,
                           u_target: np.ndarray):
    """J(f) and dJ/df by a direct forward solve and a direct adjoint solve.

    J depends on f through b(f) = R f + lifting (R = rhs_map); A is symmetric, so
    the adjoint solve is A lam = [u - u_target ; 0] and dJ/df = R^T lam."""
    b = assemble_rhs(level, f_nodal, u_dir)
    x = direct_solve(level, b)
    nv2 = 2 * level.mesh.nvel
    gvec = np.zeros_like(x)
    gvec[:nv2] = x[:nv2] - u_target.ravel()
    lam = direct_solve(level, gvec)
    grad = rhs_map(level).T @ lam
    return misfit(level, x, u_target), grad.reshape(2, level.mesh.nq, level.mesh.nq), x, lam
