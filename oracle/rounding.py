"""A-priori rounding-error bounds of one additive Vanka sweep evaluated in FP32 or BF16.

TEST INFRASTRUCTURE ONLY (like ``stokes_oracle``): the tests and the smoke check
use these bounds to compare a sweep computed in reduced precision, dof by dof,
with the FP64 oracle's sweep.  The library never imports this module.

The sweep is Algorithm 3 (Section 3.2): x_out = x + sum_i V_i^T W_i A_i^-1 V_i r
with r = b - A x and W_i = omega diag(1/m_j).  Evaluated in reduced precision,
each step adds an error that standard floating-point analysis bounds entry by
entry (u = 2^-24, the FP32 unit roundoff; u_bf = 2^-8, BF16's: 8 significant
bits, round to nearest):

  * residual: x and b are rounded to FP32 and r = b - A x is summed in FP32
    over at most 25 + 9 stencil taps per row and a few scalings, so
    |r~ - r| <= C_RES u (|b| + |A| |x|)  (gamma_n with n ~ 40, doubled);
  * BF16 patch solve (the interior patches of the tensor-core tiles):
    delta~ = fl32(bf(A^-1) bf(r~)); each product of two BF16 numbers is exact
    in FP32, both factors carry a relative error <= u_bf, and the FP32
    accumulation of 51 terms adds <= 51 u of the absolute sum, so
    |delta~ - A^-1 r~| <= (2 u_bf + u_bf^2 + 64 u) |A^-1| |r~|
                        <= (2^-7 + 2^-15) |A^-1| |r~|;
  * FP32 patch solve (block elimination with the fast-diagonalised velocity
    block): a normwise backward-stable solve, bounded componentwise by
    C_SOLVE u (|A^-1| |r| + |A^-1| |A| |delta|) -- the Oettli-Prager /
    Skeel form of a backward error C_SOLVE u |A| in the patch matrix, plus the
    forward error of the dot products of the Schur step;
  * update: x + (omega / m_j) sum of at most 9 corrections, in FP32:
    <= C_UPD u (|x| + (omega / m_j) sum |delta_i|).

The residual error propagates through the patch solve as |A^-1| times it.
The constants are generous upper estimates of the gamma_n factors; what the
tests need from them is that a plausible mistake (a wrong weight, slot, sign or
patch) gives an O(1) relative error in the dofs it touches, far above these
bounds, while correct arithmetic stays below them.
"""
from __future__ import annotations

import numpy as np

from .stokes_oracle import Level, patch_matrix

U32 = 2.0 ** -24            # FP32 unit roundoff
C_BF16 = 2.0 ** -7 + 2.0 ** -15   # BF16 x BF16 -> FP32 patch GEMM, per |A^-1| |r|
C_RES = 64.0                # FP32 residual
C_SOLVE = 512.0             # FP32 patch solve
C_UPD = 16.0                # FP32 weighted update


def sweep_error_bound(level: Level, x: np.ndarray | None, b: np.ndarray, omega: float,
                      bf16_dofs: np.ndarray | None = None) -> np.ndarray:
    """Entry-wise bound on |x_out(reduced precision) - x_out(FP64)| for one sweep.

    x None: zero initial guess.  bf16_dofs: boolean mask of the dofs whose
    corrections come from BF16 patch GEMMs (the dofs owned by tensor-core tiles);
    None means an FP32 sweep everywhere."""
    if x is None:
        x = np.zeros_like(b)
    A = level.A
    r = b - A @ x
    s_abs = np.abs(b) + abs(A) @ np.abs(x)
    nd = len(b)
    acc_bf = np.zeros(nd)     # sum_i (|A_i^-1| |r_i|)_j
    acc_res = np.zeros(nd)    # sum_i (|A_i^-1| (|b| + |A||x|)_i)_j
    acc_sk = np.zeros(nd)     # sum_i (|A_i^-1| |A_i| |delta_i|)_j
    acc_d = np.zeros(nd)      # sum_i |delta_i|_j
    dofs, cls = level.patch_dofs, level.patch_class
    for c, (slots, inv) in level.class_inv.items():
        sel = np.flatnonzero(cls == c)
        g = dofs[sel][:, slots]
        ainv = np.abs(inv)
        _, Ac = patch_matrix(A, dofs[sel[0]])
        aa = np.abs(Ac)
        R = r[g]
        D = R @ inv.T
        t_bf = np.abs(R) @ ainv.T
        t_res = s_abs[g] @ ainv.T
        t_sk = (np.abs(D) @ aa.T) @ ainv.T
        for acc, t in ((acc_bf, t_bf), (acc_res, t_res), (acc_sk, t_sk), (acc_d, np.abs(D))):
            acc += np.bincount(g.ravel(), weights=t.ravel(), minlength=nd)
    w = omega / level.mult
    bound = w * (C_RES * U32 * acc_res + C_SOLVE * U32 * (acc_bf + acc_sk)) + C_UPD * U32 * (np.abs(x) + w * acc_d)
    if bf16_dofs is not None:
        bound = bound + np.where(bf16_dofs, w * C_BF16 * acc_bf, 0.0)
    return bound


def tensor_core_dofs(n: int, tile: int = 14) -> np.ndarray:
    """Mask of the dofs whose sweep update the tensor-core kernel computes.

    Tile (bx, by) covers vertices [tile bx, tile (bx + 1)) per axis; tiles with
    1 <= bx, by <= hi, hi = (n - 2 - tile) // tile, touch only patches of the
    interior class (Section 6.3).  The kernel sweeps strips two tiles wide, so it
    takes an even number of those tiles per axis (1 .. hi, less one if the count is
    odd; none below two).  Vertex (i, j) owns the Q2 nodes (2i - 1 .. 2i) x
    (2j - 1 .. 2j) and its own pressure."""
    nq, npv = 2 * n + 1, n + 1
    hi = (n - 2 - tile) // tile if n >= 2 + 2 * tile else 0
    hi = hi - (hi % 2) if hi >= 2 else 0
    vt = np.arange(npv) // tile
    vin = (vt >= 1) & (vt <= hi)                      # per-axis vertex in a tensor-core tile
    node_owner = (np.arange(nq) + 1) // 2             # vertex owning Q2 index I on one axis
    qin = vin[node_owner]
    q2 = np.outer(qin, qin).ravel()                   # [J, I]
    p = np.outer(vin, vin).ravel()
    return np.concatenate([q2, q2, p])
