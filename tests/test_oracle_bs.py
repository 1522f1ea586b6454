"""Pins of the oracle's Braess-Sarazin relaxation (Section 3.1, Algorithm 2).

Each check is against something other than the oracle's own formula: the
exact Braess-Sarazin step it approximates (a dense solve of the block system
[[tD, B^T], [B, 0]]), the limit of many Jacobi steps, the null space of the
Schur complement, its interior rows against the vertex stencil that closed-form
1D integrals give, the multigrid contraction, and the direct solve.
"""
import numpy as np
import pytest

import stokes_inputs as si
from oracle import stokes_oracle as O


def _free_random(lv, seed):
    v = si.random_vector(lv.mesh.n, seed)
    v[lv.dmask] = 0.0
    return v


def test_exact_schur_step_is_the_exact_braess_sarazin_solve():
    """With the Schur system solved exactly, Algorithm 2's factored step equals
    omega [[tD, B^T], [B, 0]]^+ r, the original Braess-Sarazin update (Eq. bsfact):
    the velocity part exactly, the pressure part up to the constant."""
    n, t, om = 8, 1.3, 0.9
    lv = O.build_level(n, 1.0)
    nv2 = 2 * lv.mesh.nvel
    L, B, D = O.bs_blocks(lv)
    x, b = si.random_vector(n, 1), si.random_vector(n, 2)
    got = O.braess_sarazin_sweep(lv, x, b, O.BSParams(t=t, omega=om), schur="exact") - x
    K = np.block([[t * np.diag(D), B.T.toarray()], [B.toarray(), np.zeros((B.shape[0], B.shape[0]))]])
    r = b - lv.A @ x
    ref = om * np.linalg.lstsq(K, r, rcond=None)[0]
    assert np.abs(got[:nv2] - ref[:nv2]).max() <= 1e-10 * np.abs(ref[:nv2]).max()
    dp, dr = got[nv2:], ref[nv2:]
    assert np.abs((dp - dp.mean()) - (dr - dr.mean())).max() <= 1e-10 * np.abs(dr).max()


def test_schur_complement_structure():
    """S = -(1/t) B D^-1 B^T is symmetric negative semidefinite with the pressure
    constants as its kernel (B^T 1 = 0: int div psi_j = 0 for free psi_j)."""
    lv = O.build_level(8, 1.0)
    S = O.bs_schur(lv, 1.0).toarray()
    assert np.abs(S - S.T).max() <= 1e-14 * np.abs(S).max()
    assert np.abs(S @ np.ones(S.shape[0])).max() <= 1e-13 * np.abs(S).max()
    ev = np.linalg.eigvalsh(S)
    assert ev.max() <= 1e-12 * np.abs(ev).max() and np.sum(np.abs(ev) < 1e-12 * np.abs(ev).max()) == 1


def test_many_jacobi_steps_reach_the_exact_schur_solve():
    """Weighted Jacobi on S (weight 0.5) converges to the exact Schur solve for a
    consistent system: 1^T g = sum r_p (B^T 1 = 0), so the residual's pressure block
    has zero sum, as every residual of a consistent problem and its restrictions has."""
    lv = O.build_level(8, 1.0)
    nv2 = 2 * lv.mesh.nvel
    x = si.random_vector(8, 3)
    r = si.random_vector(8, 4)
    r[nv2:] -= r[nv2:].mean()
    b = lv.A @ x + r
    exact = O.braess_sarazin_sweep(lv, x, b, O.BSParams(), schur="exact")
    jac = O.braess_sarazin_sweep(lv, x, b, O.BSParams(jacobi_weight=0.5, jacobi_iters=4000))
    assert np.abs(jac[:nv2] - exact[:nv2]).max() <= 1e-8 * np.abs(exact[:nv2]).max()


def test_bs_vcycle_contraction_is_h_independent():
    rates = []
    for n in (16, 32, 64):
        H = O.build_hierarchy(n, smoother="bs")
        lv = H.levels[-1]
        nv2 = 2 * lv.mesh.nvel
        e = _free_random(lv, 5)
        e[nv2:] -= e[nv2:].mean()
        for _ in range(6):
            e2 = e - O.vcycle(H, lv.A @ e)
            e2[nv2:] -= e2[nv2:].mean()
            rate = np.linalg.norm(e2) / np.linalg.norm(e)
            e = e2
        rates.append(rate)
    assert max(rates) < 0.2 and max(rates) - min(rates) < 0.05, rates


@pytest.mark.parametrize("n", [8, 32])
def test_bs_preconditioned_fgmres_reaches_the_direct_solution(n):
    H = O.build_hierarchy(n, smoother="bs")
    lv = H.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 6), si.manufactured_velocity(n))
    res = O.solve(H, b, rtol=1e-12)
    xd = O.normalize_pressure(lv, O.direct_solve(lv, b))
    xg = O.normalize_pressure(lv, res.x)
    assert res.converged and np.linalg.norm(xg - xd) <= 1e-9 * np.linalg.norm(xd)


# ---- Schur-Uzawa (Section 3.3, Algorithm 4) ----

SU = O.BSParams(t=1.0, omega=1.0, jacobi_weight=0.4, jacobi_iters=1)   # the paper's t and Jacobi weight


def test_exact_schur_uzawa_step_is_the_block_lower_triangular_solve():
    """With the Schur system solved exactly the step is omega [[tD, 0], [B, S]]^+ r (Eq. uzblock)."""
    n, t, om = 8, 1.2, 0.8
    lv = O.build_level(n, 1.0)
    nv2 = 2 * lv.mesh.nvel
    _, B, D = O.bs_blocks(lv)
    S = O.bs_schur(lv, t).toarray()
    x, b = si.random_vector(n, 11), si.random_vector(n, 12)
    got = O.schur_uzawa_sweep(lv, x, b, O.BSParams(t=t, omega=om), schur="exact") - x
    K = np.block([[t * np.diag(D), np.zeros((nv2, S.shape[0]))], [B.toarray(), S]])
    ref = om * np.linalg.lstsq(K, b - lv.A @ x, rcond=None)[0]
    assert np.abs(got[:nv2] - ref[:nv2]).max() <= 1e-10 * np.abs(ref[:nv2]).max()
    dp, dr = got[nv2:], ref[nv2:]
    assert np.abs((dp - dp.mean()) - (dr - dr.mean())).max() <= 1e-10 * np.abs(dr).max()


def test_su_preconditioned_fgmres_reaches_the_direct_solution():
    n = 16
    H = O.build_hierarchy(n, smoother="su", bs=SU)
    lv = H.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 13), si.manufactured_velocity(n))
    res = O.solve(H, b, rtol=1e-12, maxit=300)
    xd = O.normalize_pressure(lv, O.direct_solve(lv, b))
    assert res.converged and np.linalg.norm(O.normalize_pressure(lv, res.x) - xd) <= 1e-9 * np.linalg.norm(xd)


def test_schur_complement_interior_rows_are_the_closed_form_vertex_stencil():
    """Away from the boundary S = -(1/t) B D^-1 B^T is a translation-invariant 5 x 5
    vertex stencil that follows from closed-form 1D integrals alone: Q1 hat q_a
    against the Q2 basis derivative, C(a, 2a + k) = (-1, -4, 0, 4, 1)[k + 2] / 6, and
    against the Q2 basis, N(a, 2a + k) = h (0, 1, 1, 1, 0)[k + 2] / 3 (B_x = -C (x) N,
    B_y = -N (x) C), and diag(L) = nu/90 (k m + m k) with the diagonals of the 1D Q2
    stiffness (x 1/(3h)) k = 14 / 16 and mass (x h/30) m = 8 / 16 at a vertex / midpoint
    node.  The oracle assembles B and L by quadrature; its S must equal the stencil
    (21 nonzero entries) on every vertex at distance >= 2 from the boundary."""
    c1 = {-2: -1.0, -1: -4.0, 1: 4.0, 2: 1.0}
    n1 = {-1: 1.0, 0: 1.0, 1: 1.0}
    kd = {0: 14.0, 1: 16.0}
    md = {0: 8.0, 1: 16.0}

    def wx(dI, dJ):
        return c1.get(dI, 0.0) * n1.get(dJ, 0.0)

    def wy(dI, dJ):
        return n1.get(dI, 0.0) * c1.get(dJ, 0.0)

    def s(ox, oy):
        acc = 0.0
        for nJ in range(-2, 3):
            for nI in range(-2, 3):
                mI, mJ = nI - 2 * ox, nJ - 2 * oy
                if abs(mI) > 2 or abs(mJ) > 2:
                    continue
                d = kd[nI & 1] * md[nJ & 1] + md[nI & 1] * kd[nJ & 1]
                acc += (wx(nI, nJ) * wx(mI, mJ) + wy(nI, nJ) * wy(mI, mJ)) / d
        return acc

    stencil = {(ox, oy): s(ox, oy) for ox in range(-2, 3) for oy in range(-2, 3)}
    assert sum(1 for v in stencil.values() if v != 0.0) == 21
    for n, t, nu in ((8, 1.0, 1.0), (16, 1.7, 0.3)):
        lv = O.build_level(n, nu)
        S = O.bs_schur(lv, t).toarray()
        h = 1.0 / n
        scale = -(1.0 / t) * (h / 18.0) ** 2 * (90.0 / nu)
        npv = n + 1
        for b in range(2, n - 1):
            for a in range(2, n - 1):
                v = b * npv + a
                row = np.zeros(npv * npv)
                for (ox, oy), c in stencil.items():
                    row[(b + oy) * npv + (a + ox)] = scale * c
                assert np.abs(S[v] - row).max() <= 1e-13 * np.abs(row).max(), (n, a, b)
