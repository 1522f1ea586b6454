"""Braess-Sarazin relaxation on the GPU (Section 3.1, Algorithm 2) against the
oracle: one sweep on every level (with and without an initial guess, default
and other parameters), the V-cycle, FGMRES solutions, and the mixed-FP32 form.
Tolerances as for Vanka: sweep and V-cycle 1e-12, FP64 solutions 1e-10,
mixed FP32 solutions 1e-7."""
import numpy as np
import pytest
import torch

import stokes_inputs as si
from oracle import stokes_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2401_06277_gb300 as p
    from paper_2401_06277_gb300 import build
    build.build()
    return p


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("n", [8, 16, 32])
def test_bs_sweep(pkg, n):
    from paper_2401_06277_gb300 import stokes
    H = pkg.Hierarchy(n, smoother=pkg.STOKES_SMOOTHER_BRAESS_SARAZIN)
    prm = O.BSParams()
    for l in range(H.levels):
        nl = stokes.stokes_level_n(H.handle, l)
        lv = O.build_level(nl, 1.0)
        x, b = si.random_vector(nl, 30 + l), si.random_vector(nl, 40 + l)
        got = host(H.sweep(dev(x), dev(b), level=l))
        assert rel(got, O.braess_sarazin_sweep(lv, x, b, prm)) <= 1e-12, (n, l)
        out = torch.empty(lv.mesh.ndof, dtype=torch.float64, device="cuda")
        stokes.stokes_vanka_sweep(H.handle, l, None, dev(b), out)
        assert rel(host(out), O.braess_sarazin_sweep(lv, np.zeros_like(b), b, prm)) <= 1e-12
    H.close()


def test_bs_sweep_other_parameters(pkg):
    n = 16
    prm = O.BSParams(t=1.3, omega=0.9, jacobi_weight=0.7, jacobi_iters=3)
    H = pkg.Hierarchy(n, smoother=pkg.STOKES_SMOOTHER_BRAESS_SARAZIN, bs_t=prm.t, bs_omega=prm.omega,
                      bs_jacobi_weight=prm.jacobi_weight, bs_jacobi_iters=prm.jacobi_iters)
    lv = O.build_level(n, 1.0)
    x, b = si.random_vector(n, 5), si.random_vector(n, 6)
    assert rel(host(H.sweep(dev(x), dev(b))), O.braess_sarazin_sweep(lv, x, b, prm)) <= 1e-12
    H.close()


@pytest.mark.parametrize("n", [16, 32])
def test_bs_vcycle(pkg, n):
    H = pkg.Hierarchy(n, smoother=pkg.STOKES_SMOOTHER_BRAESS_SARAZIN)
    Ho = O.build_hierarchy(n, smoother="bs")
    r = si.random_vector(n, 7)
    assert rel(host(H.vcycle(dev(r))), O.vcycle(Ho, r)) <= 1e-12
    H.close()


def test_bs_solve(pkg):
    n = 16
    H = pkg.Hierarchy(n, smoother=pkg.STOKES_SMOOTHER_BRAESS_SARAZIN, rtol=1e-13)
    lv = O.build_level(n, 1.0)
    b = O.assemble_rhs(lv, si.random_force(n, 8), si.manufactured_velocity(n))
    x, it, rr = H.solve(dev(b))
    xd = O.normalize_pressure(lv, O.direct_solve(lv, b))
    assert np.linalg.norm(O.normalize_pressure(lv, host(x)) - xd) <= 1e-10 * np.linalg.norm(xd)
    # iteration count at the default tolerance equals the oracle's
    H8 = pkg.Hierarchy(n, smoother=pkg.STOKES_SMOOTHER_BRAESS_SARAZIN)
    _, it8, _ = H8.solve(dev(b))
    assert it8 == O.solve(O.build_hierarchy(n, smoother="bs"), b).iters
    H.close()
    H8.close()


def test_bs_mixed_fp32_solution(pkg):
    n = 32
    H = pkg.Hierarchy(n, smoother=pkg.STOKES_SMOOTHER_BRAESS_SARAZIN, prec=pkg.STOKES_MIXED_FP32)
    lv = O.build_level(n, 1.0)
    b = O.assemble_rhs(lv, si.random_force(n, 9), si.manufactured_velocity(n))
    x, it, rr = H.solve(dev(b))
    xd = O.normalize_pressure(lv, O.direct_solve(lv, b))
    assert rr <= 1e-8
    assert np.linalg.norm(O.normalize_pressure(lv, host(x)) - xd) <= 1e-7 * np.linalg.norm(xd)
    H.close()


def test_bs_rejects_bf16_and_bad_parameters(pkg):
    from paper_2401_06277_gb300 import stokes
    with pytest.raises(stokes.StokesError):
        pkg.Hierarchy(16, smoother=pkg.STOKES_SMOOTHER_BRAESS_SARAZIN, prec=pkg.STOKES_MIXED_BF16)
    with pytest.raises(stokes.StokesError):
        pkg.Hierarchy(16, smoother=pkg.STOKES_SMOOTHER_BRAESS_SARAZIN, bs_jacobi_iters=0)


# ---- Schur-Uzawa (Section 3.3, Algorithm 4) ----

SU_KW = dict(bs_t=1.0, bs_omega=1.0, bs_jacobi_weight=0.4, bs_jacobi_iters=1)
SU = O.BSParams(t=1.0, omega=1.0, jacobi_weight=0.4, jacobi_iters=1)


@pytest.mark.parametrize("n", [8, 32])
def test_su_sweep_and_vcycle(pkg, n):
    from paper_2401_06277_gb300 import stokes
    H = pkg.Hierarchy(n, smoother=pkg.STOKES_SMOOTHER_SCHUR_UZAWA, **SU_KW)
    for l in range(H.levels):
        nl = stokes.stokes_level_n(H.handle, l)
        lv = O.build_level(nl, 1.0)
        x, b = si.random_vector(nl, 50 + l), si.random_vector(nl, 60 + l)
        assert rel(host(H.sweep(dev(x), dev(b), level=l)), O.schur_uzawa_sweep(lv, x, b, SU)) <= 1e-12
    Ho = O.build_hierarchy(n, smoother="su", bs=SU)
    r = si.random_vector(n, 70)
    assert rel(host(H.vcycle(dev(r))), O.vcycle(Ho, r)) <= 1e-12
    H.close()


def test_su_solve(pkg):
    n = 16
    H = pkg.Hierarchy(n, smoother=pkg.STOKES_SMOOTHER_SCHUR_UZAWA, rtol=1e-13, **SU_KW)
    lv = O.build_level(n, 1.0)
    b = O.assemble_rhs(lv, si.random_force(n, 71), si.manufactured_velocity(n))
    x, it, rr = H.solve(dev(b))
    xd = O.normalize_pressure(lv, O.direct_solve(lv, b))
    assert np.linalg.norm(O.normalize_pressure(lv, host(x)) - xd) <= 1e-10 * np.linalg.norm(xd)
    H.close()
