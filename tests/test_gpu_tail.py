"""The persistent coarse-level launch (stokes_params.tail_n) of the FP32 cycles.

The levels n <= tail_n below the finest one run the rest of the cycle (Algorithm 1:
sweeps, residuals, transfers, the exact coarse solve; V or W) as one cooperative
kernel with grid barriers between the steps.  Run with a negative tail_n, the same
kernel executes the same step list one launch per step, where kernel boundaries
order the steps: the two must agree bit for bit, which shows that every step of the
persistent launch reads what the steps before it wrote.  Against the ordinary
kernel-by-kernel path and the FP64 oracle the cycle agrees to FP32 rounding: the
same source compiled in two contexts contracts multiply-adds differently.
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


def rhs(n, seed):
    lv = O.build_level(n, 1.0)
    return lv, O.assemble_rhs(lv, si.random_force(n, seed), si.manufactured_velocity(n))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def vcycle(H, b):
    z = H.vcycle(b)
    torch.cuda.synchronize()
    return z


@pytest.mark.parametrize("cycle", [1, 2])
@pytest.mark.parametrize("n", [64, 256])
def test_persistent_launch_equals_one_launch_per_step(pkg, n, cycle):
    """Mixed FP32 form: the persistent launch (levels 4..n/2 at n = 64, 4..128 at 256)
    equals the same steps launched one by one, bit for bit, for the V- and the W-cycle,
    on two right-hand sides in a row.  The sweep configuration is pinned (8 x 8 SIMT
    tile) so the levels above the persistent launch run the same kernels in both
    hierarchies; tuned independently, they could pick differently rounding sweeps."""
    from paper_2401_06277_gb300 import stokes
    Ha = pkg.Hierarchy(n, prec=stokes.STOKES_MIXED_FP32, tile=0, tail_n=-128, cycle=cycle)
    Hb = pkg.Hierarchy(n, prec=stokes.STOKES_MIXED_FP32, tile=0, tail_n=128, cycle=cycle)
    top, steps, ctas = stokes.stokes_tail_info(Hb.handle)
    assert top == Hb.levels - 2 and steps > 0 and ctas > 0
    assert stokes.stokes_tail_info(Ha.handle)[:2] == (top, steps)
    for seed in (3, 4):
        _, b = rhs(n, seed)
        bd = dev(b)
        za, zb = vcycle(Ha, bd), vcycle(Hb, bd)
        assert torch.equal(za, zb), float((za - zb).abs().max())
    Ha.close()
    Hb.close()


@pytest.mark.parametrize("cycle", [1, 2])
def test_persistent_launch_close_to_kernel_by_kernel(pkg, cycle):
    """Against the kernel-by-kernel cycle (8 x 8 tile everywhere) and the FP64 cycle at
    256^2: the persistent launch is as close to FP64 as the kernel-by-kernel FP32 cycle
    (its difference to FP64 within 1.5x the kernel-by-kernel one, plus 1e-6), and the two
    FP32 cycles differ by FP32 rounding amplified by the cycle (<= 2e-4 of max |z|)."""
    from paper_2401_06277_gb300 import stokes
    n = 256
    Ha = pkg.Hierarchy(n, prec=stokes.STOKES_MIXED_FP32, tile=0, tail_n=0, cycle=cycle)
    Hb = pkg.Hierarchy(n, prec=stokes.STOKES_MIXED_FP32, tile=0, tail_n=128, cycle=cycle)
    H64 = pkg.Hierarchy(n, tile=0, cycle=cycle)
    _, b = rhs(n, 3)
    bd = dev(b)
    za, zb, z64 = vcycle(Ha, bd), vcycle(Hb, bd), vcycle(H64, bd)
    m = float(z64.abs().max())
    da, db = float((za - z64).abs().max()) / m, float((zb - z64).abs().max()) / m
    assert db <= 1.5 * da + 1e-6, (da, db)
    assert float((za - zb).abs().max()) / m <= 2e-4
    for H in (Ha, Hb, H64):
        H.close()


def test_persistent_launch_replaces_the_coarse_kernels(pkg):
    """At 256^2 (levels 4..128 in the persistent launch) a V(2,2) cycle is 4 sweeps,
    residual, restriction and prolongation on the finest level, the launch itself and
    the two FP64/FP32 conversions: 10 kernels."""
    from paper_2401_06277_gb300 import stokes
    H = pkg.Hierarchy(256, prec=stokes.STOKES_MIXED_FP32, tile=0, tail_n=128)
    _, b = rhs(256, 5)
    bd = dev(b)
    vcycle(H, bd)
    s0 = stokes.stokes_stats_read(H.handle)["kernel_launches"]
    vcycle(H, bd)
    assert stokes.stokes_stats_read(H.handle)["kernel_launches"] - s0 == 10
    H.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_wcycle_with_persistent_levels_against_oracle(pkg, prec):
    """W-cycle of the mixed forms (the persistent launch runs the W recursion below
    128^2) against the FP64 oracle's W-cycle, at the mixed-form bars of the V-cycle
    tests (FP32 1e-4, BF16 1e-2 of max |z|)."""
    n = 256
    H = pkg.Hierarchy(n, prec=prec, cycle=2, tail_n=128)
    Ho = O.build_hierarchy(n, gamma=2)
    lv = Ho.levels[-1]
    b = O.assemble_rhs(lv, si.random_force(n, 6), si.manufactured_velocity(n))
    z = vcycle(H, dev(b)).cpu().numpy()
    zo = O.vcycle(Ho, b)
    err = np.abs(z - zo).max() / np.abs(zo).max()
    assert err <= (1e-4 if prec == 1 else 1e-2), err
    H.close()


def test_grid_barrier_timeout_is_reported_and_recovered(pkg):
    """One CTA withholds its arrival at the first grid barrier and the barriers give
    up after 1000 polls: the other CTAs set the error flag and the kernel returns;
    stokes_device_status reports STOKES_ERR_TIMEOUT once and resets the barrier; with
    the defaults back the next cycle equals the one-launch-per-step cycle bit for bit."""
    from paper_2401_06277_gb300 import stokes
    n = 64
    H = pkg.Hierarchy(n, prec=stokes.STOKES_MIXED_FP32, tile=0, tail_n=128)
    Href = pkg.Hierarchy(n, prec=stokes.STOKES_MIXED_FP32, tile=0, tail_n=-128)
    _, b = rhs(n, 7)
    bd = dev(b)
    stokes.stokes_test_set_grid_barrier(H.handle, 1000, 0)
    z = torch.empty_like(bd)
    stokes.stokes_vcycle_apply(H.handle, bd, z)
    assert stokes.stokes_device_status(H.handle, allow_timeout=True) == stokes.STOKES_ERR_TIMEOUT
    assert stokes.stokes_device_status(H.handle) == stokes.STOKES_OK
    stokes.stokes_test_set_grid_barrier(H.handle, -1, -1)
    assert torch.equal(vcycle(H, bd), vcycle(Href, bd))
    H.close()
    Href.close()
