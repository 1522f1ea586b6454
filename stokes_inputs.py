"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds problem data only: nodal values of body forces and of the
Dirichlet velocity, evaluated at the Q2 nodes of a uniform n x n grid of the
unit square.  It contains none of the solver's arithmetic (no element
matrices, no stencils, no relaxation), so both the CPU oracle and the CUDA
path can take their inputs from here without sharing method code.

Array layout (the library's vector layout, also used by the oracle):
  Q2 nodal field  : float64 array [2, 2n+1, 2n+1], index [component, J, I],
                    node (I, J) sits at (x, y) = (I/(2n), J/(2n)).
  Q1 nodal field  : float64 array [n+1, n+1], index [j, i], vertex (i, j)
                    at (i/n, j/n).
  Stokes vector   : float64 vector [u_x (row-major, x fastest), u_y, p],
                    length 2(2n+1)^2 + (n+1)^2.

Manufactured field (the Stokes problem of Section 2.1, with the velocity
u = (sin(pi x) cos(pi y), -cos(pi x) sin(pi y)) and p = x + y - 1): the body
force is f = -nu Lap u + grad p = 2 pi^2 nu u + (1, 1).
"""
from __future__ import annotations

import numpy as np
import torch


def sizes(n: int) -> tuple[int, int, int]:
    """(Q2 nodes per axis, Q1 nodes per axis, total Stokes vector length)."""
    nq, npr = 2 * n + 1, n + 1
    return nq, npr, 2 * nq * nq + npr * npr


def _sinpi_k(k: np.ndarray, d: int) -> np.ndarray:
    """sin(pi k / d) for integers 0 <= k <= d, exact zeros at k = 0 and k = d.

    The argument is folded into [0, d/2] first (sin(pi t) = sin(pi (1 - t)))
    so that the values at both ends of the interval are exact zeros; this keeps
    the Dirichlet data's normal component exactly zero on the boundary."""
    k = np.asarray(k, dtype=np.int64)
    kk = np.minimum(k, d - k)
    return np.sin(np.pi * kk.astype(np.float64) / d)


def _cospi_k(k: np.ndarray, d: int) -> np.ndarray:
    """cos(pi k / d) = sin(pi (d/2 - k) / d) evaluated with exact zeros at k = d/2."""
    k = np.asarray(k, dtype=np.int64)
    # cos(pi t) = sin(pi (1/2 - t)); with t = k/d this is sin(pi (d - 2k) / (2d)).
    m = d - 2 * k                        # in [-d, d]
    s = np.sign(m)
    am = np.abs(m)
    return s * _sinpi_k(am, 2 * d)


def manufactured_velocity(n: int) -> np.ndarray:
    """Nodal values [2, 2n+1, 2n+1] of u = (sin pi x cos pi y, -cos pi x sin pi y)."""
    nq = 2 * n + 1
    k = np.arange(nq)
    sx, cx = _sinpi_k(k, 2 * n), _cospi_k(k, 2 * n)
    u = np.empty((2, nq, nq))
    u[0] = np.outer(cx, sx)         # [J, I]: cos(pi y_J) sin(pi x_I)
    u[1] = -np.outer(sx, cx)        # -cos(pi x_I) sin(pi y_J)
    return u


def manufactured_pressure(n: int) -> np.ndarray:
    """Q1 nodal values [n+1, n+1] of p = x + y - 1."""
    t = np.arange(n + 1) / n
    return t[:, None] + t[None, :] - 1.0


def manufactured_force(n: int, nu: float = 1.0) -> np.ndarray:
    """Nodal body force [2, 2n+1, 2n+1] for the manufactured field: 2 pi^2 nu u + (1, 1)."""
    return 2.0 * np.pi ** 2 * nu * manufactured_velocity(n) + 1.0


def polynomial_velocity(n: int) -> np.ndarray:
    """Nodal values of the divergence-free Q2 field u = (x^2, -2 x y)."""
    nq = 2 * n + 1
    t = np.arange(nq) / (2 * n)
    u = np.empty((2, nq, nq))
    u[0] = np.broadcast_to(t[None, :] ** 2, (nq, nq))
    u[1] = -2.0 * t[None, :] * t[:, None]
    return u


def polynomial_force(n: int, nu: float = 1.0) -> np.ndarray:
    """Body force for u = (x^2, -2xy), p = x + y - 1: f = (-2 nu + 1, 1)."""
    nq = 2 * n + 1
    f = np.empty((2, nq, nq))
    f[0] = -2.0 * nu + 1.0
    f[1] = 1.0
    return f


def random_force(n: int, seed: int) -> np.ndarray:
    """i.i.d. N(0, 1) nodal body force [2, 2n+1, 2n+1] from a seeded CPU generator."""
    nq = 2 * n + 1
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return torch.randn((2, nq, nq), generator=g, dtype=torch.float64).numpy()


def random_vector(n: int, seed: int) -> np.ndarray:
    """i.i.d. N(0, 1) Stokes-sized vector from a seeded CPU generator."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return torch.randn((sizes(n)[2],), generator=g, dtype=torch.float64).numpy()
