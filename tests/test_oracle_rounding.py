"""Pins of the reduced-precision sweep bound (oracle/rounding.py).

The bound is checked against sweeps emulated on the CPU in FP32 and in BF16
(round-to-nearest-even on the float32 bit pattern) and against planted mistakes:
correct reduced-precision arithmetic must stay inside it, and each mistake a
kernel could plausibly make must leave it somewhere."""
import numpy as np
import pytest

import stokes_inputs as si
from oracle import rounding as RB
from oracle import stokes_oracle as O

OMEGA = 0.7


def bf16(a):
    """float32 -> nearest BF16 (ties to even), returned as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def emulated_sweep(lv, x, b, bf16_mask):
    """Algorithm 3 in FP32; patches owning a dof in bf16_mask solve with BF16 operands."""
    A32 = lv.A.astype(np.float32)
    x32 = x.astype(np.float32)
    r = b.astype(np.float32) - A32 @ x32
    acc = np.zeros(len(b), dtype=np.float32)
    dofs, cls = lv.patch_dofs, lv.patch_class
    for c, (slots, inv) in lv.class_inv.items():
        sel = np.flatnonzero(cls == c)
        g = dofs[sel][:, slots]
        R = r[g]
        if bf16_mask is None:
            D = R @ inv.astype(np.float32).T
        else:
            D = (bf16(R) @ bf16(inv.astype(np.float32)).T).astype(np.float32)
        acc += np.bincount(g.ravel(), weights=D.ravel().astype(np.float64), minlength=len(b)).astype(np.float32)
    w = (OMEGA / lv.mult).astype(np.float32)
    return (x32 + w * acc).astype(np.float64)


@pytest.fixture(scope="module")
def lv():
    return O.build_level(32, 1.0)


@pytest.fixture(scope="module")
def xb(lv):
    x = si.random_vector(32, 3)
    b = O.assemble_rhs(lv, si.random_force(32, 4), si.manufactured_velocity(32))
    return x, b


def ratio(a, b, bound):
    """max |a - b| / bound (entries with a zero bound must agree exactly)"""
    return float(np.max(np.abs(a - b) / np.maximum(bound, 1e-300)))


def test_tensor_core_mask_counts():
    """Tiles 1..hi of 14 vertices per axis, hi = (n - 16) // 14 rounded down to an even
    count: at n = 64 (hi = 3 -> 2) tiles 1..2 hold vertices 14..41; the Q2 nodes they own
    are 2 * 14 - 1 .. 2 * 41 per axis.  At n = 128 tiles 1..8, at n = 32 none (one tile)."""
    m = RB.tensor_core_dofs(64)
    nq, npv = 129, 65
    q = m[:nq * nq].reshape(nq, nq)
    idx = np.flatnonzero(q[64])
    assert idx[0] == 27 and idx[-1] == 82 and len(idx) == 56
    assert np.array_equal(m[:nq * nq], m[nq * nq:2 * nq * nq])
    p = m[2 * nq * nq:].reshape(npv, npv)
    assert p.sum() == 28 * 28 and p[14, 14] and not p[13, 14] and p[41, 41] and not p[42, 41]
    assert RB.tensor_core_dofs(128)[2 * 257 * 257:].sum() == 112 * 112
    assert not RB.tensor_core_dofs(32).any() and not RB.tensor_core_dofs(16).any()


@pytest.mark.parametrize("zero_guess", [False, True])
def test_fp32_sweep_within_bound(lv, xb, zero_guess):
    x, b = xb
    if zero_guess:
        x = np.zeros_like(b)
    exact = O.vanka_sweep(lv, x, b, OMEGA)
    bound = RB.sweep_error_bound(lv, x, b, OMEGA)
    q = ratio(emulated_sweep(lv, x, b, None), exact, bound)
    assert q <= 1.0, q
    assert q >= 1e-4, q     # the bound is not vacuous


def test_bf16_sweep_within_bound(lv, xb):
    x, b = xb
    exact = O.vanka_sweep(lv, x, b, OMEGA)
    mask = np.ones(len(b), dtype=bool)
    bound = RB.sweep_error_bound(lv, x, b, OMEGA, bf16_dofs=mask)
    got = emulated_sweep(lv, x, b, mask)
    q = ratio(got, exact, bound)
    assert 1e-2 <= q <= 1.0, q
    # and BF16 errors are far above the FP32-only bound: the BF16 term is needed
    assert ratio(got, exact, RB.sweep_error_bound(lv, x, b, OMEGA)) > 1.0


def test_near_converged_iterate(lv, xb):
    """x near the solution: r is small against |A| |x|, the residual term dominates."""
    _, b = xb
    x = O.direct_solve(lv, b) + 1e-3 * si.random_vector(32, 5)
    exact = O.vanka_sweep(lv, x, b, OMEGA)
    bound = RB.sweep_error_bound(lv, x, b, OMEGA)
    assert ratio(emulated_sweep(lv, x, b, None), exact, bound) <= 1.0


def planted(lv, x, b, kind):
    """The FP64 sweep with one plausible kernel mistake."""
    r = b - lv.A @ x
    acc = np.zeros_like(b)
    dofs, cls = lv.patch_dofs, lv.patch_class
    w = OMEGA / lv.mult
    for c, (slots, inv) in lv.class_inv.items():
        sel = np.flatnonzero(cls == c)
        g = dofs[sel][:, slots].copy()
        D = r[g] @ inv.T
        if kind == "drop_patch" and c == 12:
            D[len(D) // 2] = 0.0
        if kind == "swap_components" and c == 12:
            k = len(D) // 3
            D[k, :25], D[k, 25:50] = D[k, 25:50].copy(), D[k, :25].copy()
        if kind == "pressure_sign" and c == 12:
            D[:, -1] = -D[:, -1]
        if kind == "slot_shift" and c == 12:
            D[:, 0:24] = D[:, 1:25].copy()
        acc += np.bincount(g.ravel(), weights=D.ravel(), minlength=len(b))
    if kind == "weight":
        w = w.copy()
        j = int(np.flatnonzero(lv.mult == 9)[len(np.flatnonzero(lv.mult == 9)) // 2])
        w[j] = OMEGA / 6.0
    return x + w * acc


@pytest.mark.parametrize("kind", ["weight", "drop_patch", "swap_components", "pressure_sign", "slot_shift"])
def test_planted_mistakes_leave_the_bound(lv, xb, kind):
    x, b = xb
    exact = O.vanka_sweep(lv, x, b, OMEGA)
    bound = RB.sweep_error_bound(lv, x, b, OMEGA, bf16_dofs=np.ones(len(b), dtype=bool))
    assert ratio(planted(lv, x, b, kind), exact, bound) > 3.0
