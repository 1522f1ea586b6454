"""Simple Vanka (per-patch inverses, Section 4 / 6.2): every patch's 51 x 51
inverse assembled and inverted on the device, stored and streamed per patch.

Checked against the oracle's per-patch sweep (each patch matrix extracted from
the assembled operator and inverted by dense LU), its V-cycle and FGMRES, and
against the shared-inverse ("tuned") GPU sweep, which computes the same
operator (tolerances as for the shared form: sweep / V-cycle 1e-12, solutions
1e-10).
"""
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
def test_simple_sweep_matches_oracle_per_patch(pkg, n):
    from paper_2401_06277_gb300 import stokes
    H = pkg.Hierarchy(n, smoother=pkg.STOKES_SMOOTHER_PER_PATCH)
    Ho = O.build_hierarchy(n, per_patch=True)
    for l in range(H.levels):
        lv = Ho.levels[l]
        x, b = si.random_vector(lv.mesh.n, 80 + l), si.random_vector(lv.mesh.n, 90 + l)
        got = host(H.sweep(dev(x), dev(b), level=l))
        ref = O.vanka_sweep(lv, x, b, 0.7)
        assert rel(got, ref) <= 1e-12, (n, l, rel(got, ref))
        out = torch.empty(lv.mesh.ndof, dtype=torch.float64, device="cuda")
        stokes.stokes_vanka_sweep(H.handle, l, None, dev(b), out)
        assert rel(host(out), O.vanka_sweep(lv, np.zeros_like(b), b, 0.7)) <= 1e-12
    H.close()


def test_simple_sweep_equals_shared_sweep(pkg):
    n = 64
    Hs = pkg.Hierarchy(n, smoother=pkg.STOKES_SMOOTHER_PER_PATCH)
    Ht = pkg.Hierarchy(n)
    x, b = dev(si.random_vector(n, 5)), dev(si.random_vector(n, 6))
    a, t = host(Hs.sweep(x, b)), host(Ht.sweep(x, b))
    assert rel(a, t) <= 1e-12
    Hs.close()
    Ht.close()


@pytest.mark.parametrize("n", [16, 32])
def test_simple_vcycle(pkg, n):
    Hs = pkg.Hierarchy(n, smoother=pkg.STOKES_SMOOTHER_PER_PATCH)
    Ho = O.build_hierarchy(n, per_patch=True)
    r = si.random_vector(n, 14)
    assert rel(host(Hs.vcycle(dev(r))), O.vcycle(Ho, r)) <= 1e-12
    Hs.close()


def test_simple_solve(pkg):
    n = 16
    Hs = pkg.Hierarchy(n, smoother=pkg.STOKES_SMOOTHER_PER_PATCH, rtol=1e-13)
    lv = O.build_level(n, 1.0)
    b = O.assemble_rhs(lv, si.random_force(n, 15), si.manufactured_velocity(n))
    x, it, rr = Hs.solve(dev(b))
    xd = O.normalize_pressure(lv, O.direct_solve(lv, b))
    xg = O.normalize_pressure(lv, host(x))
    assert np.linalg.norm(xg - xd) / np.linalg.norm(xd) <= 1e-10
    # the same iteration count as the shared-inverse smoother
    Ht = pkg.Hierarchy(n, rtol=1e-13)
    _, it_t, _ = Ht.solve(dev(b))
    assert it == it_t
    Hs.close()
    Ht.close()


def test_simple_requires_fp64(pkg):
    from paper_2401_06277_gb300 import stokes
    with pytest.raises(stokes.StokesError):
        pkg.Hierarchy(16, smoother=pkg.STOKES_SMOOTHER_PER_PATCH, prec=pkg.STOKES_MIXED_FP32)
