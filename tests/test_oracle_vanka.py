"""Pins for the oracle's additive Vanka relaxation (Section 3.2, Algorithm 3; Section 6.3)."""
import json
import os

import numpy as np
import pytest

from oracle import stokes_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("n", [4, 8, 12])
def test_patch_classes_and_sizes(n):
    facts = _golden("patch_facts.json")
    lv = O.build_level(n, 1.0)
    sizes = (lv.patch_dofs >= 0).sum(axis=1)
    assert set(np.unique(sizes)) == {facts["patch_sizes"][k] for k in ("interior", "edge", "corner")}
    # every patch of a class has the same A_i, bit for bit
    distinct = {}
    for c in np.unique(lv.patch_class):
        members = np.flatnonzero(lv.patch_class == c)
        ref = O.patch_matrix(lv.A, lv.patch_dofs[members[0]])[1]
        for k in members[1:]:
            Ai = O.patch_matrix(lv.A, lv.patch_dofs[k])[1]
            assert np.array_equal(Ai, ref)
        distinct[int(c)] = (len(members), ref)
    assert len(distinct) == facts["distinct_patch_matrices"]
    interior = [c for c, (cnt, _) in distinct.items() if c == 12]
    assert interior and distinct[12][0] == (n - 3) ** 2
    # regions: classes with both axes interior / one axis interior / none
    by_region = {"interior": 0, "edge": 0, "single": 0}
    for c in distinct:
        cy, cx = divmod(c, 5)
        k = (cx == 2) + (cy == 2)
        by_region[{2: "interior", 1: "edge", 0: "single"}[k]] += 1
    assert by_region["interior"] == facts["interior_regions"]
    assert by_region["edge"] == facts["edge_regions"]
    assert by_region["single"] == facts["single_patches"]
    # the matrices of different classes really differ (25 distinct, not fewer)
    mats = [m for _, m in distinct.values()]
    for a in range(len(mats)):
        for b in range(a + 1, len(mats)):
            assert mats[a].shape != mats[b].shape or not np.array_equal(mats[a], mats[b])


@pytest.mark.parametrize("n", [4, 8, 16, 64])
def test_table1_patch_counts(n):
    """Table 1: Form Patch RHS moves 76 + 124 l + 51 l^2 doubles; the interior-and-exterior
    inverse application reads 1520 + 3968 l + 2652 l^2 and does 2888 + 7688 l + 5202 l^2 flops."""
    t = _golden("table1_counts.json")
    ell = n - 1
    poly = lambda c: c[0] + c[1] * ell + c[2] * ell * ell
    m = O.Mesh(n)
    s = (O.patch_table(m) >= 0).sum(axis=1)          # patch sizes
    assert s.sum() == poly(t["form_patch_rhs_reads"]) == poly(t["form_patch_rhs_writes"])
    assert (s * s + s).sum() == poly(t["apply_inverse_reads"])     # matrix + rhs
    assert (2 * s * s).sum() == poly(t["apply_inverse_flops"])
    assert s.sum() == poly(t["apply_inverse_writes"])


@pytest.mark.parametrize("n", [4, 8])
def test_patch_solves_are_exact(n):
    lv = O.build_level(n, 1.0)
    rng = np.random.default_rng(0)
    for c, (slots, inv) in lv.class_inv.items():
        k = int(np.flatnonzero(lv.patch_class == c)[0])
        _, Ai = O.patch_matrix(lv.A, lv.patch_dofs[k])
        r = rng.standard_normal(len(slots))
        np.testing.assert_allclose(Ai @ (inv @ r), r, rtol=0, atol=1e-11 * np.abs(r).max())


@pytest.mark.parametrize("n", [4, 8])
def test_multiplicities(n):
    """m_j on free dofs: 9 at vertices, 6 at edge midpoints, 4 at cell centres, 1 for pressure."""
    lv = O.build_level(n, 1.0)
    m = lv.mesh
    nq = m.nq
    mult = lv.mult
    for comp in range(2):
        mm = mult[comp * m.nvel:(comp + 1) * m.nvel].reshape(nq, nq)
        for J in range(1, nq - 1):
            for I in range(1, nq - 1):
                want = (3 if I % 2 == 0 else 2) * (3 if J % 2 == 0 else 2)
                assert mm[J, I] == want
    np.testing.assert_array_equal(mult[2 * m.nvel:], 1.0)


def _sweep_brute_force(lv, x, b, omega):
    """Algorithm 3 literally: loop over patches, solve A_i d = V_i r, accumulate W_i d."""
    r = b - lv.A.toarray() @ x
    acc = np.zeros_like(x)
    for k in range(lv.patch_dofs.shape[0]):
        g = lv.patch_dofs[k][lv.patch_dofs[k] >= 0]
        Ai = lv.A.toarray()[np.ix_(g, g)]
        d = np.linalg.solve(Ai, r[g])
        acc[g] += d
    cnt = np.zeros_like(x)
    for k in range(lv.patch_dofs.shape[0]):
        g = lv.patch_dofs[k][lv.patch_dofs[k] >= 0]
        cnt[g] += 1
    return x + omega * acc / cnt


@pytest.mark.parametrize("n", [4, 8])
def test_vanka_sweep_matches_brute_force(n):
    lv = O.build_level(n, 1.0)
    rng = np.random.default_rng(n)
    x = rng.standard_normal(lv.mesh.ndof)
    b = rng.standard_normal(lv.mesh.ndof)
    got = O.vanka_sweep(lv, x, b, 0.7)
    ref = _sweep_brute_force(lv, x, b, 0.7)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_simple_and_tuned_vanka_agree():
    """Per-patch inverses ("simple" Vanka) and per-class inverses ("tuned") give the same sweep."""
    n = 8
    lt = O.build_level(n, 1.0)
    ls = O.build_level(n, 1.0, per_patch=True)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(lt.mesh.ndof)
    b = rng.standard_normal(lt.mesh.ndof)
    np.testing.assert_allclose(O.vanka_sweep(lt, x, b, 0.7), O.vanka_sweep(ls, x, b, 0.7),
                               rtol=0, atol=1e-12 * np.abs(x).max())


def test_sweep_fixed_point_is_the_solution():
    """If A x = b, a Vanka sweep leaves x unchanged (every patch residual is zero)."""
    lv = O.build_level(8, 1.0)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(lv.mesh.ndof)
    b = lv.A @ x
    np.testing.assert_allclose(O.vanka_sweep(lv, x, b, 0.7), x, rtol=0, atol=1e-12)
