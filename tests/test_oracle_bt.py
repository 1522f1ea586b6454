"""Pins of the oracle's block-triangular preconditioner (Section 3.4, Algorithm 5):
the exact-block version against a dense solve of the upper block-triangular
system, contraction of the scalar multigrid cycles on L and M, and FGMRES
reaching the direct solution."""
import numpy as np

import stokes_inputs as si
from oracle import stokes_oracle as O


def test_exact_blocks_give_the_upper_block_triangular_solve():
    n = 8
    H = O.build_hierarchy(n)
    bt = O.block_triangular_setup(H)
    lv = H.levels[-1]
    nv2 = 2 * lv.mesh.nvel
    L, B, M = bt["L"][-1].toarray(), bt["B"][-1].toarray(), bt["M"][-1].toarray()
    K = np.block([[L, B.T], [np.zeros_like(B), -M]])
    r = si.random_vector(n, 21)
    ref = np.linalg.solve(K, r)
    got = O.block_triangular_apply(H, bt, r, exact=True)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_scalar_multigrid_cycles_contract_h_independently():
    rates = {}
    prm = O.BTParams()
    for n in (16, 32):
        H = O.build_hierarchy(n)
        bt = O.block_triangular_setup(H)
        top = len(H.levels) - 1
        for name, omega, cinv in (("M", prm.omega_p, bt["Minv0"]), ("L", prm.omega_u, bt["Linv0"])):
            A = bt[name][top]
            prols = bt["PM"] if name == "M" else bt["PL"]
            e = si.random_vector(n, 22)[: A.shape[0]].copy()
            if name == "L":
                e[H.levels[top].dmask[: A.shape[0]]] = 0.0
            for _ in range(4):
                e2 = e - O.scalar_vcycle(bt[name], prols, A @ e, top, omega, prm.nu1, prm.nu2, cinv)
                rate = np.linalg.norm(e2) / np.linalg.norm(e)
                e = e2
            rates[name, n] = rate
    # weighted Jacobi of weight 0.6 (Section 6.8) on the Q1 mass matrix contracts at about
    # 0.34 per V(3,3) cycle, the velocity Laplacian (weight 1.0) at about 0.05
    assert max(rates.values()) < 0.4, rates
    assert abs(rates["M", 16] - rates["M", 32]) < 0.05 and abs(rates["L", 16] - rates["L", 32]) < 0.05, rates


def test_block_triangular_fgmres_reaches_the_direct_solution():
    n = 16
    H = O.build_hierarchy(n)
    bt = O.block_triangular_setup(H)
    lv = H.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 23), si.manufactured_velocity(n))
    res = O.fgmres(lv.A, b, np.zeros_like(b), lambda r: O.block_triangular_apply(H, bt, r), rtol=1e-12, maxit=200)
    xd = O.normalize_pressure(lv, O.direct_solve(lv, b))
    # residual 1e-12 relative; the error is larger by the conditioning of A at 16^2
    assert res.converged and np.linalg.norm(O.normalize_pressure(lv, res.x) - xd) <= 1e-8 * np.linalg.norm(xd)
