"""Pins for the oracle's multigrid (Algorithm 1), FGMRES and adjoint."""
import numpy as np
import pytest

import stokes_inputs as si
from oracle import stokes_oracle as O


def _nodal(n, fx, fy, fp):
    nq = 2 * n + 1
    t = np.arange(nq) / (2 * n)
    X, Y = np.meshgrid(t, t)
    s = np.arange(n + 1) / n
    Xp, Yp = np.meshgrid(s, s)
    return np.concatenate([fx(X, Y).ravel(), fy(X, Y).ravel(), fp(Xp, Yp).ravel()])


@pytest.mark.parametrize("nc", [4, 8])
def test_prolongation_reproduces_coarse_functions(nc):
    """P interpolates: a Q2 field vanishing on the boundary and a Q1 pressure are reproduced exactly."""
    fine, coarse = O.Mesh(2 * nc), O.Mesh(nc)
    P = O.prolongation(fine, coarse)
    ux = lambda X, Y: X * (1 - X) * Y * (1 - Y)
    uy = lambda X, Y: (X * X - X) * (2 * Y * Y - 2 * Y)
    pp = lambda X, Y: 3 * X * Y - X + 0.5
    np.testing.assert_allclose(P @ _nodal(nc, ux, uy, pp), _nodal(2 * nc, ux, uy, pp), rtol=0, atol=1e-14)
    # quarter-point weights of the 1D Q2 interpolation
    p2 = O.interp_1d_q2(nc)
    np.testing.assert_allclose(p2[1, :3], [3 / 8, 3 / 4, -1 / 8], atol=1e-15)
    np.testing.assert_allclose(p2[3, :3], [-1 / 8, 3 / 4, 3 / 8], atol=1e-15)


@pytest.mark.parametrize("nc", [4, 8])
def test_galerkin_identity(nc):
    """Nested spaces with exact quadrature: P^T A_f P = A_c on the free dofs."""
    lf, lc = O.build_level(2 * nc, 1.0), O.build_level(nc, 1.0)
    P = O.prolongation(lf.mesh, lc.mesh)
    G = (P.T @ lf.A @ P).toarray()
    free = ~lc.dmask
    np.testing.assert_allclose(G[np.ix_(free, free)], lc.A.toarray()[np.ix_(free, free)],
                               rtol=0, atol=1e-12)


def test_coarse_solve_is_exact_on_consistent_rhs():
    H = O.build_hierarchy(8)
    lv = H.levels[0]
    rng = np.random.default_rng(0)
    x = rng.standard_normal(lv.mesh.ndof)
    x[lv.dmask] = 0.0
    r = lv.A @ x
    e = O.coarse_solve(H, r)
    np.testing.assert_allclose(lv.A @ e, r, rtol=0, atol=1e-11)
    np.testing.assert_allclose(O.normalize_pressure(lv, e), O.normalize_pressure(lv, x), atol=1e-10)
    assert abs(np.ones(lv.mesh.np_ ** 2) @ (lv.Mp @ e[2 * lv.mesh.nvel:])) < 1e-13


def test_vcycle_is_linear():
    H = O.build_hierarchy(16)
    rng = np.random.default_rng(1)
    N = H.levels[-1].mesh.ndof
    r1, r2 = rng.standard_normal(N), rng.standard_normal(N)
    lhs = O.vcycle(H, 2.0 * r1 - 0.5 * r2)
    rhs = 2.0 * O.vcycle(H, r1) - 0.5 * O.vcycle(H, r2)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12 * np.abs(rhs).max())


def test_vcycle_single_level_is_coarse_solve():
    H = O.build_hierarchy(4)
    rng = np.random.default_rng(2)
    lv = H.levels[0]
    x = rng.standard_normal(lv.mesh.ndof)
    x[lv.dmask] = 0.0
    r = lv.A @ x
    np.testing.assert_allclose(lv.A @ O.vcycle(H, r), r, atol=1e-11)


def test_vcycle_contraction_is_h_independent():
    """The V(2,2) cycle as a stationary iteration contracts at a rate that does not grow with n."""
    rates = []
    for n in (8, 16, 32, 64):
        H = O.build_hierarchy(n)
        lv = H.levels[-1]
        rng = np.random.default_rng(n)
        xs = rng.standard_normal(lv.mesh.ndof)
        xs[lv.dmask] = 0.0
        b = lv.A @ xs
        x = np.zeros_like(b)
        res = [np.linalg.norm(b)]
        for _ in range(6):
            x = x + O.vcycle(H, b - lv.A @ x)
            res.append(np.linalg.norm(b - lv.A @ x))
        rates.append((res[-1] / res[2]) ** 0.25)
    assert max(rates) < 0.35, rates
    assert max(rates) < 2.0 * min(rates) + 0.05, rates


@pytest.mark.parametrize("n", [8, 16, 32])
def test_fgmres_matches_direct_solve(n):
    H = O.build_hierarchy(n)
    lv = H.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 10 + n), si.manufactured_velocity(n))
    res = O.solve(H, b, rtol=1e-12)
    assert res.converged and res.iters < 25
    xd = O.normalize_pressure(lv, O.direct_solve(lv, b))
    xs = O.normalize_pressure(lv, res.x)
    assert np.linalg.norm(xs - xd) / np.linalg.norm(xd) < 1e-9
    assert np.linalg.norm(b - lv.A @ res.x) / np.linalg.norm(b - lv.A @ O.initial_guess(lv, b)) < 1e-12


def test_fgmres_restart_and_history():
    """Small restart lengths still converge; the residual estimate is monotone within a cycle."""
    H = O.build_hierarchy(16)
    lv = H.levels[-1]
    b = O.assemble_rhs(lv, si.manufactured_force(16), si.manufactured_velocity(16))
    res = O.solve(H, b, restart=3, rtol=1e-8)
    assert res.converged
    full = O.solve(H, b, restart=30, rtol=1e-8)
    assert full.iters <= res.iters
    h = np.array(full.history)
    assert np.all(np.diff(h) <= 1e-15)


def test_fgmres_without_preconditioner_on_tiny_problem():
    """Unpreconditioned FGMRES with restart >= N is plain GMRES: it is exact after at most N steps."""
    lv = O.build_level(4, 1.0)
    A = lv.A
    rng = np.random.default_rng(5)
    xs = rng.standard_normal(lv.mesh.ndof)
    xs[lv.dmask] = 0.0
    b = A @ xs
    res = O.fgmres(A, b, np.zeros_like(b), lambda v: v, restart=lv.mesh.ndof, rtol=1e-10,
                   maxit=lv.mesh.ndof)
    assert res.converged
    np.testing.assert_allclose(A @ res.x, b, atol=1e-8)


def test_adjoint_gradient_matches_finite_differences():
    """J(f) = 1/2 ||u(f) - u_target||^2 is quadratic in f: central differences are exact up to rounding."""
    n = 8
    lv = O.build_level(n, 1.0)
    f = si.random_force(n, 7)
    ud = si.manufactured_velocity(n)
    J, g, _, _ = O.adjoint_gradient_dense(lv, f, ud, ud)
    rng = np.random.default_rng(3)
    for _ in range(4):
        d = rng.standard_normal(f.shape)
        d /= np.linalg.norm(d)
        eps = 1e-3
        Jp = O.adjoint_gradient_dense(lv, f + eps * d, ud, ud)[0]
        Jm = O.adjoint_gradient_dense(lv, f - eps * d, ud, ud)[0]
        fd = (Jp - Jm) / (2 * eps)
        an = float((g * d).sum())
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (fd, an)
    # the gradient vanishes on nodes that only touch Dirichlet rows' test functions
    assert J > 0


# ---- W-cycle (Algorithm 1 with the coarse problem cycled twice) ----

def test_wcycle_equals_vcycle_on_two_levels():
    """With the coarse level solved exactly, a second coarse cycle has nothing left to correct."""
    r = si.random_vector(8, 41)
    Hv, Hw = O.build_hierarchy(8), O.build_hierarchy(8, gamma=2)
    assert len(Hv.levels) == 2
    zv, zw = O.vcycle(Hv, r), O.vcycle(Hw, r)
    assert np.abs(zv - zw).max() <= 1e-14 * np.abs(zv).max()


def test_wcycle_contracts_at_least_as_well_and_h_independently():
    rates = {}
    for gamma in (1, 2):
        for n in (16, 32):
            H = O.build_hierarchy(n, gamma=gamma)
            lv = H.levels[-1]
            nv2 = 2 * lv.mesh.nvel
            e = si.random_vector(n, 42)
            e[lv.dmask] = 0.0
            e[nv2:] -= e[nv2:].mean()
            for _ in range(6):
                e2 = e - O.vcycle(H, lv.A @ e)
                e2[nv2:] -= e2[nv2:].mean()
                rate = np.linalg.norm(e2) / np.linalg.norm(e)
                e = e2
            rates[gamma, n] = rate
    # the asymptotic rate is set by the smoother (about 0.36 for both cycles here);
    # the second coarse correction can only make the coarse-grid error smaller
    assert rates[2, 16] <= 1.01 * rates[1, 16] and rates[2, 32] <= 1.01 * rates[1, 32], rates
    assert abs(rates[2, 16] - rates[2, 32]) < 0.05, rates


def test_wcycle_second_pass_from_the_restricted_updated_residual():
    """Restricting the fine residual after the first coarse correction gives the coarse
    residual r_c - A_c e_c (Galerkin identity), so the two-pass form equals the cycle
    on the coarse residual up to rounding."""
    n = 16
    H = O.build_hierarchy(n, gamma=2)
    lv, C = H.levels[-1], H.levels[-2]
    b = si.random_vector(n, 43)
    x = O.relax(H, lv, np.zeros_like(b), b)
    rc = lv.P.T @ (b - lv.A @ x)
    e1 = O.vcycle(H, rc, len(H.levels) - 2)
    x1 = x + lv.P @ e1
    rc2 = lv.P.T @ (b - lv.A @ x1)
    ref = rc - C.A @ e1
    assert np.abs(rc2 - ref).max() <= 1e-12 * np.abs(ref).max()
