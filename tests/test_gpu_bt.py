"""Block-triangular preconditioner on the GPU (Section 3.4, Algorithm 5) against
the oracle: one application (three V(3,3) cycles of scalar multigrid on M, then
on L; tolerance 1e-12 as for the V-cycle) and FGMRES with it."""
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
def test_bt_application(pkg, n):
    H = pkg.Hierarchy(n, precond=1)
    Ho = O.build_hierarchy(n)
    bt = O.block_triangular_setup(Ho)
    for seed in (81, 82):
        r = si.random_vector(n, seed)
        assert rel(host(H.vcycle(dev(r))), O.block_triangular_apply(Ho, bt, r)) <= 1e-12, (n, seed)
    H.close()


def test_bt_fgmres(pkg):
    n = 16
    H = pkg.Hierarchy(n, precond=1, rtol=1e-12)
    Ho = O.build_hierarchy(n)
    bt = O.block_triangular_setup(Ho)
    lv = Ho.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 83), si.manufactured_velocity(n))
    x, it, rr = H.solve(dev(b))
    xd = O.normalize_pressure(lv, O.direct_solve(lv, b))
    assert np.linalg.norm(O.normalize_pressure(lv, host(x)) - xd) <= 1e-8 * np.linalg.norm(xd)
    H8 = pkg.Hierarchy(n, precond=1)
    _, it8, rr8 = H8.solve(dev(b))
    ref = O.fgmres(lv.A, b, O.initial_guess(lv, b), lambda r: O.block_triangular_apply(Ho, bt, r))
    assert rr8 <= 1e-8 and it8 == ref.iters
    H.close()
    H8.close()


def test_bt_requires_fp64(pkg):
    from paper_2401_06277_gb300 import stokes
    with pytest.raises(stokes.StokesError):
        pkg.Hierarchy(16, precond=1, prec=pkg.STOKES_MIXED_FP32)
