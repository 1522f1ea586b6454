"""Parity at the benchmark's full size (2048 x 2048 elements, 10 levels) in the launch
configuration bench.py times (the same hierarchy parameters and autotuned tiles).

The oracle cannot assemble a 2048^2 problem, but one Vanka sweep, the operator and
the grid transfers are local: a dof's output depends only on data within a few
nodes.  A random pattern that vanishes outside a box in the middle of a 32^2 grid
(and its Dirichlet margins) is embedded at an even node offset deep inside the
2048^2 grid; there the GPU result must equal the oracle's 32^2 result element by
element, after one exact rescaling: the velocity block L is independent of h in
2D while B scales with h (Eq. 4), so with D = diag(I_u, s I_p) and s = h_big / h_small
= 32 / 2048 (a power of two, exact in floating point) the big operator restricted
to the window is D A_small D, and one additive Vanka sweep, whose patch matrices are
R_i D A D R_i^T, satisfies  sweep_big(x, b) = D^-1 sweep_small(D x, D^-1 b).  The full
solve is checked through properties that hold at any size: the true FP64 residual
and the nodal error of the manufactured solution.
"""
import numpy as np
import pytest
import torch

import stokes_inputs as si
from oracle import stokes_oracle as O

pytestmark = pytest.mark.gpu

NBIG = 2048
NS = 32          # small grid of the oracle
OFF = 1400       # vertex offset of the small grid inside the big one (Q2 offset 2 * OFF)


@pytest.fixture(scope="module")
def big():
    import paper_2401_06277_gb300 as pkg
    from paper_2401_06277_gb300 import build
    build.build()
    H = pkg.Hierarchy(NBIG, rtol=1e-8, restart=30)
    yield H
    H.close()


def pattern(n, seed, box=(12, 20)):
    """Random x with support in vertices [box) and Q2 nodes [2 box), zero elsewhere."""
    rng = np.random.default_rng(seed)
    nq, npr = 2 * n + 1, n + 1
    u = np.zeros((2, nq, nq))
    p = np.zeros((npr, npr))
    a, b = box
    u[:, 2 * a: 2 * b, 2 * a: 2 * b] = rng.standard_normal((2, 2 * (b - a), 2 * (b - a)))
    p[a:b, a:b] = rng.standard_normal((b - a, b - a))
    return np.concatenate([u.ravel(), p.ravel()])


def embed(v_small, n_small, n_big, off):
    """Place a small-grid vector at vertex offset `off` (Q2 offset 2 off) in a zero big-grid vector."""
    nqs, nps, nqb, npb = 2 * n_small + 1, n_small + 1, 2 * n_big + 1, n_big + 1
    us = v_small[: 2 * nqs * nqs].reshape(2, nqs, nqs)
    ps = v_small[2 * nqs * nqs:].reshape(nps, nps)
    ub = np.zeros((2, nqb, nqb))
    pb = np.zeros((npb, npb))
    ub[:, 2 * off: 2 * off + nqs, 2 * off: 2 * off + nqs] = us
    pb[off: off + nps, off: off + nps] = ps
    return np.concatenate([ub.ravel(), pb.ravel()])


def window(v_big, n_small, n_big, off):
    nqs, nps, nqb, npb = 2 * n_small + 1, n_small + 1, 2 * n_big + 1, n_big + 1
    ub = v_big[: 2 * nqb * nqb].reshape(2, nqb, nqb)
    pb = v_big[2 * nqb * nqb:].reshape(npb, npb)
    return np.concatenate([ub[:, 2 * off: 2 * off + nqs, 2 * off: 2 * off + nqs].ravel(),
                           pb[off: off + nps, off: off + nps].ravel()])


def outside_norm(v_big, n_small, n_big, off):
    """Largest magnitude outside the embedded window."""
    nqs, nps, nqb, npb = 2 * n_small + 1, n_small + 1, 2 * n_big + 1, n_big + 1
    ub = v_big[: 2 * nqb * nqb].reshape(2, nqb, nqb).copy()
    pb = v_big[2 * nqb * nqb:].reshape(npb, npb).copy()
    ub[:, 2 * off: 2 * off + nqs, 2 * off: 2 * off + nqs] = 0.0
    pb[off: off + nps, off: off + nps] = 0.0
    return max(np.abs(ub).max(), np.abs(pb).max())


S = NS / NBIG    # h_big / h_small, exactly 2^-6


def pscale(x, n, f):
    """D x with D = diag(I_u, f I_p) on an n^2 grid vector."""
    y = x.copy()
    y[2 * (2 * n + 1) ** 2:] *= f
    return y


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def cpu(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_fullsize_operator(big):
    lv = O.build_level(NS, 1.0)
    xs = pattern(NS, 1)
    ref = pscale(lv.A @ pscale(xs, NS, S), NS, S)
    y = cpu(big.apply(gpu(embed(xs, NS, NBIG, OFF))))
    err = np.abs(window(y, NS, NBIG, OFF) - ref).max() / np.abs(ref).max()
    assert err <= 1e-13, err
    assert outside_norm(y, NS, NBIG, OFF) == 0.0


def test_fullsize_vanka_sweep(big):
    """One FP64 sweep on the finest 2048^2 level, with the tile shape the bench uses."""
    lv = O.build_level(NS, 1.0)
    xs, bs = pattern(NS, 2), pattern(NS, 3)
    ref = pscale(O.vanka_sweep(lv, pscale(xs, NS, S), pscale(bs, NS, 1 / S), 0.7), NS, 1 / S)
    out = cpu(big.sweep(gpu(embed(xs, NS, NBIG, OFF)), gpu(embed(bs, NS, NBIG, OFF))))
    err = np.abs(window(out, NS, NBIG, OFF) - ref).max() / np.abs(ref).max()
    assert err <= 1e-12, err
    assert outside_norm(out, NS, NBIG, OFF) == 0.0


@pytest.mark.parametrize("prec", [1, 2])
def test_fullsize_mixed_sweep_within_rounding_bound(prec):
    """One sweep of the mixed FP32 (prec 1) and BF16 (prec 2) forms on the finest 2048^2
    level, in the bench's configuration: the autotuned strip sweep on the interior, where
    the window sits (vertex offset 1400, inside the strips' tiles 1..144).  Every dof of the
    window is within the rounding bound of oracle/rounding.py, evaluated on the 32^2 problem
    for the scaled inputs and mapped back by D^-1 (the scaling is by powers of two, so the
    rounding errors scale with it exactly, barring underflow); outside the window the output
    is zero.  In the BF16 form the error exceeds the FP32-only bound somewhere in the window:
    the tensor cores produced it."""
    import paper_2401_06277_gb300 as pkg
    from oracle import rounding as RB
    from paper_2401_06277_gb300 import stokes
    H = pkg.Hierarchy(NBIG, rtol=1e-8, restart=30, prec=prec)
    assert stokes.stokes_level_tile(H.handle, H.levels - 1) == 3, "the tuner did not pick the strip sweep"
    lv = O.build_level(NS, 1.0)
    xs, bs = pattern(NS, 6 + prec), pattern(NS, 8 + prec)
    xsc, bsc = pscale(xs, NS, S), pscale(bs, NS, 1 / S)
    ref = pscale(O.vanka_sweep(lv, xsc, bsc, 0.7), NS, 1 / S)
    out = cpu(H.relax(gpu(embed(xs, NS, NBIG, OFF)), gpu(embed(bs, NS, NBIG, OFF))))
    H.close()
    allbf = np.ones_like(bs, dtype=bool) if prec == 2 else None
    bound = pscale(RB.sweep_error_bound(lv, xsc, bsc, 0.7, bf16_dofs=allbf), NS, 1 / S)
    got = window(out, NS, NBIG, OFF)
    q = np.max(np.abs(got - ref) / np.maximum(bound, 1e-300))
    assert q <= 1.0, q
    assert outside_norm(out, NS, NBIG, OFF) == 0.0
    if prec == 2:
        fp32 = pscale(RB.sweep_error_bound(lv, xsc, bsc, 0.7), NS, 1 / S)
        assert np.max(np.abs(got - ref) / np.maximum(fp32, 1e-300)) > 1.0


def test_fullsize_transfers(big):
    """Restriction and prolongation between the two finest levels (2048 -> 1024)."""
    from paper_2401_06277_gb300 import stokes
    lf, lc = O.build_level(2 * NS, 1.0), O.build_level(NS, 1.0)
    P = O.prolongation(lf.mesh, lc.mesh)
    L = big.levels - 1
    offc = 700  # coarse vertex offset in the 1024 grid; the fine window sits at 2 offc in the 2048 grid
    # restriction of a fine pattern
    rf = pattern(2 * NS, 4, box=(24, 40))
    rc_ref = P.T @ rf
    rc = torch.zeros(si.sizes(NBIG // 2)[2], dtype=torch.float64, device="cuda")
    stokes.stokes_restrict(big.handle, L, gpu(embed(rf, 2 * NS, NBIG, 2 * offc)), rc)
    rc = cpu(rc)
    assert np.abs(window(rc, NS, NBIG // 2, offc) - rc_ref).max() <= 1e-13 * np.abs(rc_ref).max()
    assert outside_norm(rc, NS, NBIG // 2, offc) == 0.0
    # prolongation of a coarse pattern
    ec = pattern(NS, 5)
    xf = torch.zeros(si.sizes(NBIG)[2], dtype=torch.float64, device="cuda")
    stokes.stokes_prolong_add(big.handle, L, gpu(embed(ec, NS, NBIG // 2, offc)), xf)
    xf = cpu(xf)
    ref = P @ ec
    assert np.abs(window(xf, 2 * NS, NBIG, 2 * offc) - ref).max() <= 1e-13 * np.abs(ref).max()
    assert outside_norm(xf, 2 * NS, NBIG, 2 * offc) == 0.0


def test_fullsize_manufactured_solve(big):
    """FGMRES + V(2,2) at 2048^2 on the manufactured field: true FP64 residual <= 1e-8 of the
    initial one, nodal velocity error and (mean-free) pressure error small."""
    n = NBIG
    f = gpu(si.manufactured_force(n))
    ud = gpu(si.manufactured_velocity(n))
    b = big.assemble_rhs(f, ud)
    x, it, rr = big.solve(b)
    assert rr <= 1e-8 and it <= 12
    # the true residual through a second kernel (the allocation-free residual norm; it
    # shares the operator kernel's stencil coefficient tables, not its tiling or code)
    from paper_2401_06277_gb300 import stokes
    x0 = torch.empty_like(b)
    stokes.stokes_initial_guess(big.handle, b, x0)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    stokes.stokes_residual_norm_noalloc(n, 1.0, b, x, nrm)
    r_end = float(nrm.item())
    stokes.stokes_residual_norm_noalloc(n, 1.0, b, x0, nrm)
    assert r_end <= 1.01e-8 * float(nrm.item()), (r_end, float(nrm.item()))
    xv = cpu(x)
    nq = 2 * n + 1
    ue = si.manufactured_velocity(n).ravel()
    eu = np.abs(xv[: 2 * nq * nq] - ue).max()
    p = xv[2 * nq * nq:]
    pe = si.manufactured_pressure(n).ravel()
    ep = np.abs((p - p.mean()) - (pe - pe.mean())).max()
    print(f"2048^2 manufactured: it={it} rr={rr:.3e} true={r_end / float(nrm.item()):.3e} "
          f"max|u-u_e|={eu:.3e} max|p-p_e|={ep:.3e}")
    assert eu <= 1e-6, eu
    assert ep <= 1e-4, ep


def _zero_mean_diff(x, ref, n):
    p0 = 2 * (2 * n + 1) ** 2
    a, r = x.clone(), ref.clone()
    a[p0:] -= a[p0:].mean()
    r[p0:] -= r[p0:].mean()
    return float((a - r).abs().max() / r.abs().max())


def test_fullsize_mixed_solutions_as_accurate_as_fp64(big):
    """The mixed FP32 / BF16 forms at 2048^2 on the manufactured problem, stopped at the
    same 1e-8 residual as the FP64 form.  Two iterations stopped at 1e-8 differ by the
    operator's conditioning times 1e-8 (here ~1e-6), whatever their precision, so each is
    measured against an FP64 solve to 1e-11: the mixed solutions must be as accurate as the
    FP64 one (within twice its error, plus 1e-8)."""
    import paper_2401_06277_gb300 as pkg
    n = NBIG
    f = gpu(si.manufactured_force(n))
    ud = gpu(si.manufactured_velocity(n))
    b = big.assemble_rhs(f, ud)
    x64, _, _ = big.solve(b)
    Href = pkg.Hierarchy(n, rtol=1e-11, restart=30)
    xref, _, rr = Href.solve(b)
    Href.close()
    assert rr <= 1e-11
    e64 = _zero_mean_diff(x64, xref, n)
    for prec in (1, 2):
        Hm = pkg.Hierarchy(n, rtol=1e-8, restart=30, prec=prec)
        xm, it, rr = Hm.solve(b)
        Hm.close()
        em, d = _zero_mean_diff(xm, xref, n), _zero_mean_diff(xm, x64, n)
        print(f"2048^2 prec {prec}: iters {it}, error vs 1e-11 solve {em:.3e} (FP64 at 1e-8: {e64:.3e}), "
              f"difference to the FP64 form {d:.3e}")
        assert rr <= 1e-8 and em <= 2.0 * e64 + 1e-8, (prec, em, e64)


def test_fullsize_mixed_gap_is_the_tolerance(big):
    """The benchmark's 2048^2 problem (N(0,1) nodal force, seed 0) solved in FP64, mixed
    FP32 and mixed BF16 at rtol 1e-8 and 1e-10, and in FP64 at 1e-11.  Two solves stopped
    at a residual tolerance differ by up to the operator's conditioning times that
    tolerance, so the gap between a mixed solution and the FP64 one must shrink with the
    tolerance: at rtol 1e-10 both mixed solutions are within 1e-7 (max norm, relative,
    pressures at zero mean) of the FP64 solution at 1e-10.  The table is printed."""
    import paper_2401_06277_gb300 as pkg
    n = NBIG
    f = gpu(si.random_force(n, 0))
    ud = gpu(si.manufactured_velocity(n))
    b = big.assemble_rhs(f, ud)
    sol = {}
    for prec in (0, 1, 2):
        for rtol in (1e-8, 1e-10):
            H = pkg.Hierarchy(n, rtol=rtol, restart=30, prec=prec)
            x, it, rr = H.solve(b)
            H.close()
            assert rr <= rtol, (prec, rtol, rr)
            sol[(prec, rtol)] = (x, it)
    H = pkg.Hierarchy(n, rtol=1e-11, restart=30)
    xref, _, rr = H.solve(b)
    H.close()
    assert rr <= 1e-11
    names = {0: "FP64", 1: "FP32", 2: "BF16"}
    rows = []
    for rtol in (1e-8, 1e-10):
        x64 = sol[(0, rtol)][0]
        for prec in (0, 1, 2):
            x, it = sol[(prec, rtol)]
            d = _zero_mean_diff(x, x64, n)
            e = _zero_mean_diff(x, xref, n)
            rows.append((rtol, names[prec], it, d, e))
    print("\nrtol   form  iters  diff-to-FP64-same-rtol  diff-to-FP64-1e-11")
    for rtol, nm, it, d, e in rows:
        print(f"{rtol:.0e}  {nm}  {it:5d}  {d:22.3e}  {e:18.3e}")
    for rtol, nm, it, d, e in rows:
        if rtol == 1e-10 and nm != "FP64":
            assert d <= 1e-7, (nm, d)
    # the gap shrinks with the tolerance
    for prec in (1, 2):
        d8 = _zero_mean_diff(sol[(prec, 1e-8)][0], sol[(0, 1e-8)][0], n)
        d10 = _zero_mean_diff(sol[(prec, 1e-10)][0], sol[(0, 1e-10)][0], n)
        assert d10 <= 0.1 * d8, (prec, d8, d10)
