"""Pins for the oracle's discretisation (Section 2): element matrices, operator, RHS.

Every check here compares the oracle against something other than itself:
closed-form 1D matrices typed from the textbook formulas, exact symmetry,
polynomial exactness, the divergence-free interpolant, and convergence rates.
"""
import numpy as np
import pytest

import stokes_inputs as si
from oracle import stokes_oracle as O

# Closed-form 1D matrices on one element of length h (local nodes 0, h/2, h for
# Q2; 0, h for Q1).  Stiffness/mass are the standard quadratic-element ones.
K1 = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 3.0          # times 1/h
M1 = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 30.0           # times h
C1 = np.array([[-5, 4, 1], [-1, -4, 5]]) / 6.0                        # int q_a Q_c'
N1 = np.array([[1, 2, 0], [0, 2, 1]]) / 6.0                           # int q_a Q_c, times h
P1 = np.array([[2, 1], [1, 2]]) / 6.0                                 # Q1 mass, times h


@pytest.mark.parametrize("h", [1.0, 0.25, 1.0 / 64])
def test_element_matrices_match_tensor_products(h):
    em = O.element_matrices(h)
    K, M = K1 / h, M1 * h
    # local index b*3 + a (y index b, x index a) -> kron(y-factor, x-factor)
    np.testing.assert_allclose(em["stiff"], np.kron(M, K) + np.kron(K, M), rtol=0, atol=1e-13)
    np.testing.assert_allclose(em["mass"], np.kron(M, M), rtol=0, atol=1e-15 * max(1, h * h))
    # b(v, p) = -int p div v
    np.testing.assert_allclose(em["bx"], -np.kron(N1 * h, C1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(em["by"], -np.kron(C1, N1 * h), rtol=0, atol=1e-15)
    np.testing.assert_allclose(em["pmass"], np.kron(P1 * h, P1 * h), rtol=0, atol=1e-16)


@pytest.mark.parametrize("n", [4, 8])
def test_operator_exactly_symmetric(n):
    lv = O.build_level(n, 1.0)
    D = (lv.A - lv.A.T).tocoo()
    assert np.all(D.data == 0.0)
    # Dirichlet rows are identity rows
    d = np.flatnonzero(lv.dmask)
    sub = lv.A[d]
    assert np.all(sub.getnnz(axis=1) == 1)
    np.testing.assert_array_equal(lv.A.diagonal()[d], 1.0)


@pytest.mark.parametrize("n", [4, 8])
def test_row_and_column_sums(n):
    K, M, Bx, By, Mp = O.assemble_blocks(O.Mesh(n))
    # constants lie in the kernel of the (unconstrained) stiffness
    assert np.abs(K @ np.ones(K.shape[1])).max() < 1e-12
    # sum_k B_kj = -int div psi_j = 0 for interior velocity nodes
    nq = 2 * n + 1
    inner = np.zeros((nq, nq), dtype=bool)
    inner[1:-1, 1:-1] = True
    cs_x = np.asarray(Bx.sum(axis=0)).ravel()[inner.ravel()]
    cs_y = np.asarray(By.sum(axis=0)).ravel()[inner.ravel()]
    assert np.abs(cs_x).max() < 1e-15 and np.abs(cs_y).max() < 1e-15
    # total mass is the area of the unit square
    assert abs(M.sum() - 1.0) < 1e-13 and abs(Mp.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("n", [4, 8, 16])
def test_polynomial_solution_is_reproduced_exactly(n):
    """u = (x^2, -2xy) in Q2, p = x + y - 1 in Q1: the discrete solution is the interpolant."""
    lv = O.build_level(n, 1.0)
    u = si.polynomial_velocity(n)
    b = O.assemble_rhs(lv, si.polynomial_force(n), u)
    x = O.normalize_pressure(lv, O.direct_solve(lv, b))
    ref = np.concatenate([u[0].ravel(), u[1].ravel(), si.manufactured_pressure(n).ravel()])
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-10)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_manufactured_interpolant_is_discretely_divergence_free(n):
    lv = O.build_level(n, 1.0)
    m = lv.mesh
    u = si.manufactured_velocity(n)
    Bu = lv.A_full[2 * m.nvel:, : 2 * m.nvel] @ np.concatenate([u[0].ravel(), u[1].ravel()])
    assert np.abs(Bu).max() < 1e-15


@pytest.mark.parametrize("n", [4, 8, 16])
def test_rhs_is_consistent(n):
    """The pressure rows of b sum to zero, so b is orthogonal to ker A = (0, 1_p)."""
    lv = O.build_level(n, 1.0)
    m = lv.mesh
    for f in (si.manufactured_force(n), si.random_force(n, 3)):
        b = O.assemble_rhs(lv, f, si.manufactured_velocity(n))
        assert abs(b[2 * m.nvel:].sum()) < 1e-14
        assert np.all(b[lv.dmask] == np.concatenate([si.manufactured_velocity(n)[0].ravel(),
                                                     si.manufactured_velocity(n)[1].ravel()])[lv.dmask[: 2 * m.nvel]])


def test_convergence_rates():
    """O(h^3) velocity and (at least) O(h^2) pressure L2 errors for the sin/cos field."""
    ue = lambda X, Y: (np.sin(np.pi * X) * np.cos(np.pi * Y), -np.cos(np.pi * X) * np.sin(np.pi * Y))
    pe = lambda X, Y: X + Y - 1.0
    eu, ep = [], []
    for n in (8, 16, 32):
        lv = O.build_level(n, 1.0)
        b = O.assemble_rhs(lv, si.manufactured_force(n), si.manufactured_velocity(n))
        x = O.normalize_pressure(lv, O.direct_solve(lv, b))
        a, c = O.l2_errors(lv, x, ue, pe)
        eu.append(a)
        ep.append(c)
    ru = np.log2(np.array(eu[:-1]) / np.array(eu[1:]))
    rp = np.log2(np.array(ep[:-1]) / np.array(ep[1:]))
    assert np.all(ru > 2.9), ru
    assert np.all(rp > 1.9), rp
    assert eu[-1] < 1e-5


def test_viscosity_scales_velocity_block_only():
    lv1 = O.build_level(8, 1.0)
    lv2 = O.build_level(8, 2.5)
    m = lv1.mesh
    nv2 = 2 * m.nvel
    d = ~lv1.dmask
    A1 = lv1.A_full.toarray()
    A2 = lv2.A_full.toarray()
    np.testing.assert_allclose(A2[:nv2, :nv2], 2.5 * A1[:nv2, :nv2], rtol=1e-14, atol=1e-14)
    np.testing.assert_array_equal(A2[nv2:, :nv2], A1[nv2:, :nv2])
    assert d.sum() > 0
