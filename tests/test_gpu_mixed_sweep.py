"""Mixed-precision sweeps dof by dof against the FP64 oracle, and the failure paths.

stokes_relaxation_sweep runs one sweep of the V-cycle's smoother in the
hierarchy's arithmetic: FP32 (mixed form; with tile 3 the interior tiles on the
FP32 strip kernel) or FP32 with the interior patch solves as BF16 tensor-core
GEMMs (BF16 form).  Each output dof is compared with
the oracle's FP64 sweep (Algorithm 3) against the a-priori rounding bound of
oracle/rounding.py, computed from the oracle's own patch inverses and residual:
BF16 terms on the dofs that tensor-core tiles own, FP32 terms everywhere.
"""
import numpy as np
import pytest
import torch

import stokes_inputs as si
from oracle import rounding as RB
from oracle import stokes_oracle as O

pytestmark = pytest.mark.gpu

OMEGA = 0.7
_LV = {}


def level(n):
    if n not in _LV:
        _LV[n] = O.build_level(n, 1.0)
    return _LV[n]


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


def ratio(got, ref, bound):
    return float(np.max(np.abs(got - ref) / np.maximum(bound, 1e-300)))


def inputs(n, seed, zero_guess):
    lv = level(n)
    b = O.assemble_rhs(lv, si.random_force(n, seed), si.manufactured_velocity(n))
    x = None if zero_guess else si.random_vector(n, seed + 1)
    return lv, x, b


def gpu_relax(H, x, b, lvl=None):
    return host(H.relax(None if x is None else dev(x), dev(b), level=lvl))


@pytest.mark.parametrize("zero_guess", [False, True])
@pytest.mark.parametrize("n", [64, 128])
def test_bf16_tensor_core_sweep_dof_by_dof(pkg, n, zero_guess):
    """Tile 3: the interior 14 x 14 tiles on the tensor cores, the ring on the FP32 SIMT
    kernel.  Every dof within its bound; on the dofs the tensor-core tiles own, the error
    is above the FP32-only bound, so BF16 arithmetic (the tcgen05 kernel) produced them."""
    from paper_2401_06277_gb300 import stokes
    H = pkg.Hierarchy(n, prec=stokes.STOKES_MIXED_BF16, tile=3)
    lv, x, b = inputs(n, 50 + n, zero_guess)
    got = gpu_relax(H, x, b)
    ref = O.vanka_sweep(lv, np.zeros_like(b) if x is None else x, b, OMEGA)
    tc = RB.tensor_core_dofs(n)
    assert tc.any()
    bound = RB.sweep_error_bound(lv, x, b, OMEGA, bf16_dofs=tc)
    q = ratio(got, ref, bound)
    assert q <= 1.0, q
    fp32_only = RB.sweep_error_bound(lv, x, b, OMEGA)
    assert ratio(got[tc], ref[tc], fp32_only[tc]) > 1.0
    assert ratio(got[~tc], ref[~tc], fp32_only[~tc]) <= 1.0     # the ring is FP32
    H.close()


def test_bf16_sweep_on_a_coarser_level(pkg):
    """Level n = 64 of a 128 hierarchy (tensor-core tiles 1..2)."""
    from paper_2401_06277_gb300 import stokes
    H = pkg.Hierarchy(128, prec=stokes.STOKES_MIXED_BF16, tile=3)
    lv, x, b = inputs(64, 77, False)
    got = gpu_relax(H, x, b, lvl=H.levels - 2)
    ref = O.vanka_sweep(lv, x, b, OMEGA)
    assert ratio(got, ref, RB.sweep_error_bound(lv, x, b, OMEGA, bf16_dofs=RB.tensor_core_dofs(64))) <= 1.0
    H.close()


@pytest.mark.parametrize("tile", [-1, 0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("n", [32, 64])
def test_fp32_sweep_dof_by_dof(pkg, n, tile):
    """The mixed FP32 form's sweep, every tile configuration, within the FP32 bound."""
    from paper_2401_06277_gb300 import stokes
    H = pkg.Hierarchy(n, prec=stokes.STOKES_MIXED_FP32, tile=tile)
    for zero_guess in (False, True):
        lv, x, b = inputs(n, 90 + n + tile, zero_guess)
        got = gpu_relax(H, x, b)
        ref = O.vanka_sweep(lv, np.zeros_like(b) if x is None else x, b, OMEGA)
        q = ratio(got, ref, RB.sweep_error_bound(lv, x, b, OMEGA))
        assert q <= 1.0, (zero_guess, q)
    H.close()


@pytest.mark.parametrize("zero_guess", [False, True])
@pytest.mark.parametrize("n", [64, 128, 256])
def test_fp32_strip_sweep_dof_by_dof(pkg, n, zero_guess):
    """Tile 3 in the mixed FP32 form: the interior 14 x 14 tiles on the strip kernel, each
    patch solved in FP32 by fast diagonalisation, the ring on the SIMT kernel.  Every dof,
    those of the strips included, within the FP32 bound."""
    from paper_2401_06277_gb300 import stokes
    H = pkg.Hierarchy(n, prec=stokes.STOKES_MIXED_FP32, tile=3)
    lv, x, b = inputs(n, 130 + n, zero_guess)
    got = gpu_relax(H, x, b)
    ref = O.vanka_sweep(lv, np.zeros_like(b) if x is None else x, b, OMEGA)
    assert RB.tensor_core_dofs(n).any()
    q = ratio(got, ref, RB.sweep_error_bound(lv, x, b, OMEGA))
    assert q <= 1.0, q
    H.close()


def test_fp32_strip_sweep_on_a_coarser_level_and_its_launches(pkg):
    """Level n = 128 of a 256 hierarchy within the FP32 bound; a sweep with strips is two
    kernels (strip and ring) and three FP64/FP32 conversions, one without (the SIMT 8 x 8
    tile, tile 0) is one kernel and the conversions."""
    from paper_2401_06277_gb300 import stokes
    H = pkg.Hierarchy(256, prec=stokes.STOKES_MIXED_FP32, tile=3)
    lv, x, b = inputs(128, 79, False)
    got = gpu_relax(H, x, b, lvl=H.levels - 2)
    ref = O.vanka_sweep(lv, x, b, OMEGA)
    assert ratio(got, ref, RB.sweep_error_bound(lv, x, b, OMEGA)) <= 1.0
    xd, bd = dev(x), dev(b)
    out = torch.empty_like(bd)
    for tile, launches in ((3, 5), (0, 4)):
        Ht = pkg.Hierarchy(128, prec=stokes.STOKES_MIXED_FP32, tile=tile)
        torch.cuda.synchronize()
        s0 = stokes.stokes_stats_read(Ht.handle)
        stokes.stokes_relaxation_sweep(Ht.handle, Ht.levels - 1, xd, bd, out)
        s1 = stokes.stokes_stats_read(Ht.handle)
        assert s1["kernel_launches"] - s0["kernel_launches"] == launches, tile
        assert s1["tc_launches"] == s0["tc_launches"]   # no tensor-core kernel in the FP32 form
        Ht.close()
    H.close()


def test_bf16_form_launches_the_tensor_core_kernel(pkg):
    """The library's counters: one relaxation sweep on the 128^2 level with tile 3 is the
    tensor-core kernel plus its SIMT ring (2 launches) and three FP64/FP32 conversions; a
    V(2,2) cycle launches the tensor-core kernel 4 times on each level with at least two
    interior tiles per axis (128 and 64: 8 launches); with the persistent coarse-level
    launch for n <= 64 (tail_n = 64, the SIMT tile there) only on 128: 4."""
    from paper_2401_06277_gb300 import stokes
    H = pkg.Hierarchy(128, prec=stokes.STOKES_MIXED_BF16, tile=3, tail_n=64)
    lv, x, b = inputs(128, 5, False)
    xd, bd = dev(x), dev(b)
    out = torch.empty_like(bd)
    torch.cuda.synchronize()
    s0 = stokes.stokes_stats_read(H.handle)
    stokes.stokes_relaxation_sweep(H.handle, H.levels - 1, xd, bd, out)
    s1 = stokes.stokes_stats_read(H.handle)
    assert s1["tc_launches"] - s0["tc_launches"] == 1
    assert s1["kernel_launches"] - s0["kernel_launches"] == 5
    stokes.stokes_vcycle_apply(H.handle, bd, out)
    s2 = stokes.stokes_stats_read(H.handle)
    assert s2["tc_launches"] - s1["tc_launches"] == 4
    H.close()
    H = pkg.Hierarchy(128, prec=stokes.STOKES_MIXED_BF16, tile=3, tail_n=0)
    torch.cuda.synchronize()
    s1 = stokes.stokes_stats_read(H.handle)
    stokes.stokes_vcycle_apply(H.handle, bd, out)
    s2 = stokes.stokes_stats_read(H.handle)
    assert s2["tc_launches"] - s1["tc_launches"] == 8
    H.close()


def test_expired_device_wait_is_reported_and_recovered(pkg):
    """The tensor-core kernel's first bounded wait is given 0 polls: it expires, the kernel
    sets the error flag, waits for its bulk copy with the full limit and exits.  FGMRES
    returns STOKES_ERR_TIMEOUT; stokes_device_status reports a V-cycle's expiry once; with
    the default limit restored the same hierarchy solves correctly."""
    from paper_2401_06277_gb300 import stokes
    n = 64
    H = pkg.Hierarchy(n, prec=stokes.STOKES_MIXED_BF16, tile=3)
    lv = level(n)
    b = O.assemble_rhs(lv, si.random_force(n, 8), si.manufactured_velocity(n))
    bd = dev(b)
    stokes.stokes_test_set_wait_limit(H.handle, 0)
    with pytest.raises(stokes.StokesError) as ei:
        H.solve(bd)
    assert ei.value.status == stokes.STOKES_ERR_TIMEOUT
    assert stokes.stokes_device_status(H.handle) == stokes.STOKES_OK   # reported once
    z = torch.empty_like(bd)
    stokes.stokes_vcycle_apply(H.handle, bd, z)
    assert stokes.stokes_device_status(H.handle, allow_timeout=True) == stokes.STOKES_ERR_TIMEOUT
    assert stokes.stokes_device_status(H.handle) == stokes.STOKES_OK
    stokes.stokes_test_set_wait_limit(H.handle, -1)
    x, it, rr = H.solve(bd)
    assert rr <= 1e-8
    xo = O.normalize_pressure(lv, O.direct_solve(lv, b))
    xg = O.normalize_pressure(lv, host(x))
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-6
    H.close()


def test_allocation_failure_returns_oom_and_frees(pkg):
    """A cap on the bytes one creation may allocate makes stokes_hierarchy_create fail
    with STOKES_ERR_OOM part-way (after the level vectors, before the Krylov basis); what
    it had allocated is freed, and without the cap the same creation succeeds."""
    from paper_2401_06277_gb300 import stokes
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        stokes.stokes_test_set_alloc_limit(64 << 20)
        for _ in range(3):
            with pytest.raises(stokes.StokesError) as ei:
                pkg.Hierarchy(256)
            assert ei.value.status == stokes.STOKES_ERR_OOM
    finally:
        stokes.stokes_test_set_alloc_limit(0)
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] <= (16 << 20)
    H = pkg.Hierarchy(256)
    assert H.levels == 7
    H.close()
