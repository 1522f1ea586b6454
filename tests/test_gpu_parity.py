"""GPU parity: every step of the hot path through the C ABI against the FP64 CPU oracle.

Sizes span several 8 x 8 vertex tiles with ragged tails (n + 1 vertices per
axis is never a multiple of 8).  Tolerances are relative to the largest
magnitude of the reference: operator 1e-13, Vanka sweep and V-cycle 1e-12,
FGMRES solutions 1e-10 (pressure normalised to zero mean on both sides).
"""
import numpy as np
import pytest
import torch

import stokes_inputs as si
from oracle import stokes_oracle as O

pytestmark = pytest.mark.gpu

_ORACLE = {}


def oracle_h(n):
    if n not in _ORACLE:
        _ORACLE[n] = O.build_hierarchy(n)
    return _ORACLE[n]


@pytest.fixture(scope="module")
def pkg():
    import paper_2401_06277_gb300 as p
    from paper_2401_06277_gb300 import build
    build.build()
    return p


_GPU = {}


def gpu_h(pkg, n, **kw):
    key = (n, tuple(sorted(kw.items())))
    if key not in _GPU:
        _GPU[key] = pkg.Hierarchy(n, **kw)
    return _GPU[key]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def rvec(n, seed, dirichlet_zero=False, lv=None):
    v = si.random_vector(n, seed)
    if dirichlet_zero:
        v[lv.dmask] = 0.0
    return v


@pytest.mark.parametrize("n", [4, 8, 16, 32, 64])
def test_operator_and_residual(pkg, n):
    H = gpu_h(pkg, n)
    Ho = oracle_h(n)
    lv = Ho.levels[-1]
    x, b = rvec(n, 1), rvec(n, 2)
    y = host(H.apply(dev(x)))
    assert rel(y, lv.A @ x) <= 1e-13
    r = host(H.residual(dev(b), dev(x)))
    assert rel(r, b - lv.A @ x) <= 1e-13
    # every level of the hierarchy
    for l in range(H.levels - 1):
        nl = H.level_n(l)
        xl = rvec(nl, 10 + l)
        assert rel(host(H.apply(dev(xl), level=l)), Ho.levels[l].A @ xl) <= 1e-13


@pytest.mark.parametrize("n", [4, 8, 32])
@pytest.mark.parametrize("force", ["manufactured", "random"])
def test_rhs_assembly(pkg, n, force):
    H = gpu_h(pkg, n)
    lv = oracle_h(n).levels[-1]
    f = si.manufactured_force(n) if force == "manufactured" else si.random_force(n, 5)
    ud = si.manufactured_velocity(n)
    b = host(H.assemble_rhs(dev(f), dev(ud)))
    bo = O.assemble_rhs(lv, f, ud)
    assert rel(b, bo) <= 1e-13
    assert abs(b[2 * lv.mesh.nvel:].sum()) <= 1e-14 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("n", [4, 8, 16, 32, 64])
def test_vanka_sweep(pkg, n):
    from paper_2401_06277_gb300 import stokes
    H = gpu_h(pkg, n)
    Ho = oracle_h(n)
    for l in range(H.levels):
        lv = Ho.levels[l]
        nl = lv.mesh.n
        x, b = rvec(nl, 3 + l), rvec(nl, 4 + l)
        got = host(H.sweep(dev(x), dev(b), level=l))
        ref = O.vanka_sweep(lv, x, b, 0.7)
        assert rel(got, ref) <= 1e-12, (n, l, rel(got, ref))
        # zero initial guess (x = NULL in the ABI)
        out = torch.empty(lv.mesh.ndof, dtype=torch.float64, device="cuda")
        stokes.stokes_vanka_sweep(H.handle, l, None, dev(b), out)
        ref0 = O.vanka_sweep(lv, np.zeros_like(b), b, 0.7)
        assert rel(host(out), ref0) <= 1e-12


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("n", [8, 32, 64])
def test_vanka_sweep_tile_shapes(pkg, n, tile):
    """Every configuration of the FP64 sweep gives the same sweep: fused tiles of 8x8, 16x8,
    16x16 and 14x14 vertices, and the split sweep (own-patch solves writing the corrections,
    then the update kernel)."""
    from paper_2401_06277_gb300 import stokes
    H = gpu_h(pkg, n, tile=tile)
    assert stokes.stokes_level_tile(H.handle, H.levels - 1) == tile
    Ho = oracle_h(n)
    for l in (H.levels - 1, max(H.levels - 2, 0)):
        lv = Ho.levels[l]
        x, b = rvec(lv.mesh.n, 50 + l), rvec(lv.mesh.n, 60 + l)
        assert rel(host(H.sweep(dev(x), dev(b), level=l)), O.vanka_sweep(lv, x, b, 0.7)) <= 1e-12
    r = rvec(n, 70)
    assert rel(host(H.vcycle(dev(r))), O.vcycle(Ho, r)) <= 1e-12


def test_vanka_sweep_rejects_aliasing(pkg):
    from paper_2401_06277_gb300 import stokes
    H = gpu_h(pkg, 8)
    x = dev(rvec(8, 1))
    with pytest.raises(stokes.StokesError):
        stokes.stokes_vanka_sweep(H.handle, H.levels - 1, x, x, x)


@pytest.mark.parametrize("n", [8, 16, 64])
def test_restrict_and_prolong(pkg, n):
    from paper_2401_06277_gb300 import stokes
    H = gpu_h(pkg, n)
    Ho = oracle_h(n)
    for l in range(1, H.levels):
        P = Ho.levels[l].P
        nf, nc = Ho.levels[l].mesh.n, Ho.levels[l - 1].mesh.n
        rf = rvec(nf, 20 + l)
        rc = torch.empty(si.sizes(nc)[2], dtype=torch.float64, device="cuda")
        stokes.stokes_restrict(H.handle, l, dev(rf), rc)
        assert rel(host(rc), P.T @ rf) <= 1e-13
        ec = rvec(nc, 30 + l)
        xf = rvec(nf, 40 + l)
        xt = dev(xf)
        stokes.stokes_prolong_add(H.handle, l, dev(ec), xt)
        assert rel(host(xt), xf + P @ ec) <= 1e-13


def test_coarse_solve(pkg):
    from paper_2401_06277_gb300 import stokes
    H = gpu_h(pkg, 16)
    Ho = oracle_h(16)
    lv = Ho.levels[0]
    x = rvec(4, 9, dirichlet_zero=True, lv=lv)
    r = lv.A @ x
    e = torch.empty_like(dev(r))
    stokes.stokes_coarse_solve(H.handle, dev(r), e)
    assert rel(host(e), O.coarse_solve(Ho, r)) <= 1e-12
    # a consistent right-hand side is solved exactly, with int p = 0
    assert rel(lv.A @ host(e), r) <= 1e-11


@pytest.mark.parametrize("n", [4, 8, 16, 32, 64])
def test_vcycle(pkg, n):
    H = gpu_h(pkg, n)
    Ho = oracle_h(n)
    lv = Ho.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 11), si.manufactured_velocity(n))
    z = host(H.vcycle(dev(b)))
    zo = O.vcycle(Ho, b)
    assert rel(z, zo) <= 1e-12, rel(z, zo)
    r = rvec(n, 12)
    assert rel(host(H.vcycle(dev(r))), O.vcycle(Ho, r)) <= 1e-12


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (0, 2), (3, 0)])
def test_vcycle_sweep_counts(pkg, nu1, nu2):
    n = 16
    H = gpu_h(pkg, n, nu1=nu1, nu2=nu2)
    Ho = O.build_hierarchy(n, nu1=nu1, nu2=nu2)
    r = rvec(n, 13)
    assert rel(host(H.vcycle(dev(r))), O.vcycle(Ho, r)) <= 1e-12


@pytest.mark.parametrize("orth", [0, 2])
@pytest.mark.parametrize("n", [8, 16, 32, 64])
def test_fgmres_solution(pkg, n, orth):
    """orth 0 on these grids is classical Gram-Schmidt (DGKS); orth 2 forces the
    modified form that grids of 2^20 dofs and more take by default."""
    H = gpu_h(pkg, n, orth=orth)
    Ho = oracle_h(n)
    lv = Ho.levels[-1]
    f = si.manufactured_force(n) if n == 32 else si.random_force(n, 100 + n)
    ud = si.manufactured_velocity(n)
    b = O.assemble_rhs(lv, f, ud)
    x, it, rr = H.solve(dev(b))
    xg = O.normalize_pressure(lv, host(x))
    res = O.solve(Ho, b)
    xo = O.normalize_pressure(lv, res.x)
    assert rr <= 1e-8 and res.converged
    assert it == res.iters
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10
    # the true residual recomputed on the CPU
    r0 = np.linalg.norm(b - lv.A @ O.initial_guess(lv, b))
    assert np.linalg.norm(b - lv.A @ host(x)) / r0 <= 1.01e-8


@pytest.mark.parametrize("orth", [1, 2])
def test_fgmres_against_direct_solve(pkg, orth):
    n = 16
    H = gpu_h(pkg, n, rtol=1e-13, orth=orth)
    lv = oracle_h(n).levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 7), si.manufactured_velocity(n))
    x, it, rr = H.solve(dev(b))
    xd = O.normalize_pressure(lv, O.direct_solve(lv, b))
    xg = O.normalize_pressure(lv, host(x))
    assert np.linalg.norm(xg - xd) / np.linalg.norm(xd) <= 1e-10


@pytest.mark.parametrize("orth", [1, 2])
def test_fgmres_small_restart_and_maxit(pkg, orth):
    from paper_2401_06277_gb300 import stokes
    n = 16
    lv = oracle_h(n).levels[-1]
    b = O.assemble_rhs(lv, si.manufactured_force(n), si.manufactured_velocity(n))
    H3 = gpu_h(pkg, n, restart=3, orth=orth)
    x, it, rr = H3.solve(dev(b))
    ref = O.solve(O.build_hierarchy(n), b, restart=3)
    assert it == ref.iters and rr <= 1e-8
    H1 = gpu_h(pkg, n, maxit=2)
    x, it, rr = H1.solve(dev(b), allow_not_converged=True)
    assert it == 2 and rr > 1e-8
    with pytest.raises(stokes.StokesError) as e:
        H1.solve(dev(b))
    assert e.value.status == stokes.STOKES_NOT_CONVERGED


def test_fgmres_rejects_nonfinite_rhs(pkg):
    from paper_2401_06277_gb300 import stokes
    n = 8
    H = gpu_h(pkg, n)
    lv = oracle_h(n).levels[-1]
    b = O.assemble_rhs(lv, si.manufactured_force(n), si.manufactured_velocity(n))
    b[lv.mesh.nvel + 40] = np.nan
    with pytest.raises(stokes.StokesError) as e:
        H.solve(dev(b))
    assert e.value.status == stokes.STOKES_ERR_NONFINITE


def test_zero_rhs_returns_zero(pkg):
    n = 8
    H = gpu_h(pkg, n)
    b = torch.zeros(si.sizes(n)[2], dtype=torch.float64, device="cuda")
    x, it, rr = H.solve(b)
    assert it == 0 and float(x.abs().max()) == 0.0


@pytest.mark.parametrize("nu", [0.01, 3.0])
def test_viscosity(pkg, nu):
    n = 16
    H = gpu_h(pkg, n, viscosity=nu)
    Ho = O.build_hierarchy(n, nu=nu)
    r = rvec(n, 17)
    assert rel(host(H.apply(dev(r))), Ho.levels[-1].A @ r) <= 1e-13
    assert rel(host(H.vcycle(dev(r))), O.vcycle(Ho, r)) <= 1e-12


def test_adjoint_gradient(pkg):
    n = 16
    H = gpu_h(pkg, n, rtol=1e-12)
    lv = oracle_h(n).levels[-1]
    f = si.random_force(n, 7)
    ud = si.manufactured_velocity(n)
    J, grad_o, x_o, lam_o = O.adjoint_gradient_dense(lv, f, ud, ud)
    b = H.assemble_rhs(dev(f), dev(ud))
    x, _, _ = H.solve(b)
    g = x.clone()
    nv2 = 2 * lv.mesh.nvel
    g[:nv2] -= dev(ud.ravel())
    g[nv2:] = 0.0
    lam, grad, it, rr = H.adjoint(g)
    grad = host(grad).reshape(grad_o.shape)
    assert rel(grad, grad_o) <= 1e-9


# ---------------------------------------------------------------------------
# Mixed-precision preconditioner (FP32 vectors, residuals and patch solves;
# FGMRES and the coarse solve in FP64)
# ---------------------------------------------------------------------------
MIXED = {}


def mixed_h(pkg, n, **kw):
    from paper_2401_06277_gb300 import stokes
    return gpu_h(pkg, n, prec=stokes.STOKES_MIXED_FP32, **kw)


@pytest.mark.parametrize("tile", [-1, 4, 5, 6])
@pytest.mark.parametrize("n", [8, 32, 64])
def test_mixed_vcycle_close_to_fp64(pkg, n, tile):
    """The FP32 V-cycle agrees with the FP64 oracle's V-cycle to FP32 rounding.

    Bar 1e-4 relative to max |z|: FP32 unit roundoff (6e-8) amplified by the
    cancellation in b - A x after the pre-sweeps (|A x| / |r| up to ~1e2) and
    compounded over up to five levels.  The mixed form is held to the
    solution bar (1e-7 after FP64 FGMRES to 1e-8), tested below.  tile -1: tuned;
    4 / 5: the split FP32 sweep on every level."""
    H = mixed_h(pkg, n, tile=tile)
    Ho = oracle_h(n)
    lv = Ho.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 21), si.manufactured_velocity(n))
    err = rel(host(H.vcycle(dev(b))), O.vcycle(Ho, b))
    MIXED[("vcycle", n)] = err
    assert err <= 1e-4, err


@pytest.mark.parametrize("tile,orth", [(-1, 0), (5, 0), (-1, 2)])
@pytest.mark.parametrize("n", [16, 64])
def test_mixed_fgmres_solution(pkg, n, tile, orth):
    """FGMRES (FP64) with the FP32 preconditioner reaches the same 1e-8 residual; the
    solution is within 1e-7 of the FP64 oracle's solution at the same tolerance."""
    H = mixed_h(pkg, n, tile=tile, orth=orth)
    Ho = oracle_h(n)
    lv = Ho.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 31), si.manufactured_velocity(n))
    x, it, rr = H.solve(dev(b))
    res = O.solve(Ho, b)
    xg = O.normalize_pressure(lv, host(x))
    xo = O.normalize_pressure(lv, res.x)
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    MIXED[("fgmres", n)] = (err, it, res.iters)
    assert rr <= 1e-8
    r0 = np.linalg.norm(b - lv.A @ O.initial_guess(lv, b))
    assert np.linalg.norm(b - lv.A @ host(x)) / r0 <= 1.01e-8
    assert it <= res.iters + 2
    assert err <= 1e-7, err


# ---------------------------------------------------------------------------
# BF16 tensor-core form (interior patch solves as tcgen05 GEMMs, FP32 vectors)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("tile", [3, -1])
@pytest.mark.parametrize("n", [32, 64, 128])
def test_bf16_vcycle_close_to_fp64(pkg, n, tile):
    """BF16 patch GEMMs: the V-cycle agrees with the FP64 oracle's to BF16 rounding.
    tile 3 forces the tensor-core sweep on every level where it fits; -1 lets the
    autotuner choose between it and the SIMT shapes per level.

    Bar 1e-2 relative to max |z|: BF16 keeps 8 significant bits (unit roundoff
    2^-9 = 2e-3) in both the gathered residuals and the patch inverse, the
    products are accumulated in FP32."""
    from paper_2401_06277_gb300 import stokes
    H = gpu_h(pkg, n, prec=stokes.STOKES_MIXED_BF16, tile=tile)
    Ho = oracle_h(n)
    lv = Ho.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 21), si.manufactured_velocity(n))
    err = rel(host(H.vcycle(dev(b))), O.vcycle(Ho, b))
    assert err <= 1e-2, err


@pytest.mark.parametrize("tile,orth", [(3, 0), (-1, 0), (3, 2)])
@pytest.mark.parametrize("n", [64, 128])
def test_bf16_fgmres_solution(pkg, n, tile, orth):
    """FGMRES (FP64) with the BF16 tensor-core preconditioner: same 1e-8 residual,
    solution within 1e-7 of the FP64 oracle's at the same tolerance."""
    from paper_2401_06277_gb300 import stokes
    H = gpu_h(pkg, n, prec=stokes.STOKES_MIXED_BF16, tile=tile, orth=orth)
    Ho = oracle_h(n)
    lv = Ho.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 41), si.manufactured_velocity(n))
    x, it, rr = H.solve(dev(b))
    res = O.solve(Ho, b)
    xg = O.normalize_pressure(lv, host(x))
    xo = O.normalize_pressure(lv, res.x)
    assert rr <= 1e-8 and it <= res.iters + 2
    r0 = np.linalg.norm(b - lv.A @ O.initial_guess(lv, b))
    assert np.linalg.norm(b - lv.A @ host(x)) / r0 <= 1.01e-8
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-7


def test_bf16_uses_the_tensor_core_kernel(pkg):
    """With tile 3 the finest 128^2 level sweeps its interior tiles on the tensor cores
    and the ring on the 14x14 SIMT tile: a finest-level sweep is two launches (the
    tensor-core kernel and the ring), one of them the tensor-core kernel."""
    from paper_2401_06277_gb300 import stokes
    H = gpu_h(pkg, 128, prec=stokes.STOKES_MIXED_BF16, tile=3)
    assert stokes.stokes_level_tile(H.handle, H.levels - 1) == 3
    b = dev(si.random_vector(128, 3))
    out = torch.empty_like(b)
    torch.cuda.synchronize()
    s0 = stokes.stokes_stats_read(H.handle)
    stokes.stokes_relaxation_sweep(H.handle, H.levels - 1, None, b, out)   # zero guess: b -> FP32, sweep, widen
    s1 = stokes.stokes_stats_read(H.handle)
    assert s1["tc_launches"] - s0["tc_launches"] == 1
    assert s1["kernel_launches"] - s0["kernel_launches"] == 2 + 2


# ---------------------------------------------------------------------------
# Differentiation: torch.autograd through the solve, backward = adjoint solve
# ---------------------------------------------------------------------------
def _misfit(x, ut, nv2):
    d = x[:nv2] - ut
    return 0.5 * torch.dot(d, d)


def test_autograd_gradient_matches_dense_adjoint(pkg):
    """dJ/df from the autograd backward equals the oracle's direct-solve adjoint (16 x 16)."""
    n = 16
    H = gpu_h(pkg, n, rtol=1e-13)
    lv = oracle_h(n).levels[-1]
    f0 = si.random_force(n, 7)
    ud = si.manufactured_velocity(n)
    J_o, g_o, _, _ = O.adjoint_gradient_dense(lv, f0, ud, ud)
    f = dev(f0).requires_grad_(True)
    x = pkg.stokes_solve(f, dev(ud), H)
    J = _misfit(x, dev(ud).reshape(-1), 2 * lv.mesh.nvel)
    J.backward()
    assert abs(J.item() - J_o) <= 1e-9 * J_o
    assert rel(host(f.grad), g_o) <= 1e-9


def test_autograd_gradient_matches_finite_differences_512(pkg):
    """512 x 512, J(f) = 1/2 ||u(f) - u_target||^2 (u_target the manufactured velocity, f
    seeded N(0,1)): the adjoint gradient along 16 random unit directions matches central
    differences within 1e-5 relative.

    J is exactly quadratic in f, so a central difference has no truncation error at any
    step; the step only trades against rounding.  With J ~ 3e4 and |grad J . d| ~ 1e-3 a
    step of 1e-6 leaves the difference below the rounding noise of J in FP64
    (1e-16 J / 2e-6 ~ 1e-6 absolute, plus solver noise), so the step is 1.  The FD solves
    run to 1e-10 (the FP64 floor of the relative residual at 512^2 is ~1e-11)."""
    n = 512
    H = gpu_h(pkg, n, rtol=1e-10)
    nv2 = 2 * (2 * n + 1) ** 2
    ud = dev(si.manufactured_velocity(n))
    ut = ud.reshape(-1)
    f = dev(si.random_force(n, 7)).requires_grad_(True)
    J = _misfit(pkg.stokes_solve(f, ud, H), ut, nv2)
    J.backward()
    g = f.grad.detach()
    eps = 1.0
    worst = 0.0
    for k in range(16):
        d = dev(si.random_force(n, 100 + k))
        d /= torch.linalg.vector_norm(d)
        with torch.no_grad():
            xp = pkg.stokes_solve(f.detach() + eps * d, ud, H)
            xm = pkg.stokes_solve(f.detach() - eps * d, ud, H)
            # J(f+) - J(f-) = 1/2 (u+ - u-) . (u+ + u- - 2 u_target), no cancellation of J values
            dJ = 0.5 * torch.dot(xp[:nv2] - xm[:nv2], xp[:nv2] + xm[:nv2] - 2 * ut)
        fd = float(dJ / (2 * eps))
        an = float((g * d).sum())
        worst = max(worst, abs(fd - an) / max(abs(an), 1e-30))
    assert worst <= 1e-5, worst


def test_adjoint_projects_inconsistent_pressure_data(pkg):
    """A gradient with a pressure component along ker A^T is projected, not rejected."""
    n = 16
    H = gpu_h(pkg, n, rtol=1e-12)
    lv = oracle_h(n).levels[-1]
    g = rvec(n, 90, dirichlet_zero=True, lv=lv)
    lam, grad, it, rr = H.adjoint(dev(g))
    gp = g.copy()
    gp[2 * lv.mesh.nvel:] -= gp[2 * lv.mesh.nvel:].mean()
    assert rr <= 1e-12
    assert rel(lv.A @ host(lam), gp) <= 1e-10


# ---------------------------------------------------------------------------
# Batched form: problems of uneven size in lockstep, one CUDA graph per iteration
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 2])
def test_batch_uneven_sizes_match_single_solves(pkg, prec):
    """A batch of problems of different sizes gives, problem by problem, the single-solve
    result (same iterations, <= 1e-12), and each problem's solution is the FP64 oracle's
    FGMRES solution of that problem (<= 1e-10 in FP64, <= 1e-7 for the mixed forms, the
    solution bars at rtol 1e-8)."""
    from paper_2401_06277_gb300 import stokes
    ns = [16, 64, 32, 64] if prec == 0 else [32, 128, 64]
    # BF16: tensor-core and SIMT sweeps round differently, so both sides fix the configuration
    kw = {"tile": 3} if prec == 2 else {}
    B = pkg.Batch(ns, prec=prec, **kw)
    rhs, refs = [], []
    for k, n in enumerate(ns):
        f = dev(si.random_force(n, 500 + k))
        ud = dev(si.manufactured_velocity(n))
        rhs.append(B.assemble_rhs(k, f, ud))
        H = gpu_h(pkg, n, prec=prec, **kw)
        x, it, rr = H.solve(H.assemble_rhs(f, ud))
        refs.append((host(x), it))
    xs, its, rels = B.solve(rhs)
    oracle_res = {}
    for k, n in enumerate(ns):
        Ho = oracle_h(n)
        lv = Ho.levels[-1]
        assert its[k] == refs[k][1]
        assert rels[k] <= 1e-8
        xb = O.normalize_pressure(lv, host(xs[k]))
        xr = O.normalize_pressure(lv, refs[k][0])
        assert np.linalg.norm(xb - xr) / np.linalg.norm(xr) <= 1e-12
        bo = O.assemble_rhs(lv, si.random_force(n, 500 + k), si.manufactured_velocity(n))
        if (n, k) not in oracle_res:
            oracle_res[(n, k)] = O.normalize_pressure(lv, O.solve(Ho, bo).x)
        xo = oracle_res[(n, k)]
        assert np.linalg.norm(xb - xo) / np.linalg.norm(xo) <= (1e-10 if prec == 0 else 1e-7)
    B.close()


@pytest.mark.parametrize("orth", [0, 2])
def test_batch_many_rhs_one_grid(pkg, orth):
    """Eight right-hand sides on one grid (FP32 preconditioner): every solve reaches 1e-8
    and matches the oracle's solution within 1e-7, with either Gram-Schmidt captured in
    the batch's per-iteration graphs."""
    from paper_2401_06277_gb300 import stokes
    n = 32
    ns = [n] * 8
    B = pkg.Batch(ns, prec=stokes.STOKES_MIXED_FP32, restart=12, orth=orth)
    Ho = oracle_h(n)
    lv = Ho.levels[-1]
    rhs, bo = [], []
    for k in range(8):
        f = si.random_force(n, 2000 + k)
        ud = si.manufactured_velocity(n)
        bo.append(O.assemble_rhs(lv, f, ud))
        rhs.append(B.assemble_rhs(k, dev(f), dev(ud)))
    xs, its, rels = B.solve(rhs)
    for k in range(8):
        assert rels[k] <= 1e-8
        xo = O.normalize_pressure(lv, O.solve(Ho, bo[k]).x)
        xg = O.normalize_pressure(lv, host(xs[k]))
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-7
    B.close()


@pytest.mark.parametrize("smoother", [0, 2])
@pytest.mark.parametrize("n", [16, 32])
def test_wcycle(pkg, n, smoother):
    """W-cycle (two coarse-grid corrections per level) with Vanka or Braess-Sarazin relaxation."""
    H = pkg.Hierarchy(n, cycle=2, smoother=smoother)
    Ho = O.build_hierarchy(n, gamma=2, smoother="bs" if smoother == 2 else "vanka")
    r = rvec(n, 44)
    assert rel(host(H.vcycle(dev(r))), O.vcycle(Ho, r)) <= 1e-12
    lv = Ho.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 45), si.manufactured_velocity(n))
    x, it, rr = H.solve(dev(b))
    assert rr <= 1e-8 and it == O.solve(Ho, b).iters
    H.close()
