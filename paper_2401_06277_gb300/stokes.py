"""Thin Python binding of the C ABI in include/stokes_vanka.h (argument marshalling only).

Every function here has the name of the C entry point it calls and forwards
device pointers of torch tensors; all arithmetic runs in the CUDA library.
If the library has not been built (``paper_2401_06277_gb300.build``), loading
fails with an error: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

STOKES_OK = 0
STOKES_ERR_ARG = 1
STOKES_ERR_OOM = 2
STOKES_ERR_CUDA = 3
STOKES_ERR_NONFINITE = 4
STOKES_NOT_CONVERGED = 5
STOKES_ERR_TIMEOUT = 6

STOKES_FP64 = 0
STOKES_MIXED_FP32 = 1
STOKES_MIXED_BF16 = 2
STOKES_SMOOTHER_SHARED = 0
STOKES_SMOOTHER_PER_PATCH = 1
STOKES_SMOOTHER_BRAESS_SARAZIN = 2
STOKES_SMOOTHER_SCHUR_UZAWA = 3

_STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_NONFINITE",
           5: "NOT_CONVERGED", 6: "ERR_TIMEOUT"}


class StokesError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class stokes_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("vcycles", ctypes.c_longlong),
                ("sweeps_timed", ctypes.c_longlong), ("sweep_ms", ctypes.c_double),
                ("tc_launches", ctypes.c_longlong)]


class stokes_params(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("omega", ctypes.c_double),
                ("coarse_n", ctypes.c_int), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("rtol", ctypes.c_double), ("prec", ctypes.c_int), ("tile", ctypes.c_int),
                ("smoother", ctypes.c_int), ("bs_t", ctypes.c_double), ("bs_omega", ctypes.c_double),
                ("bs_jacobi_weight", ctypes.c_double), ("bs_jacobi_iters", ctypes.c_int),
                ("cycle", ctypes.c_int), ("precond", ctypes.c_int), ("bt_cycles", ctypes.c_int),
                ("bt_nu", ctypes.c_int), ("bt_omega_u", ctypes.c_double), ("bt_omega_p", ctypes.c_double),
                ("tail_n", ctypes.c_int), ("orth", ctypes.c_int)]


_lib = None


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is not built; run paper_2401_06277_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, D, VP = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    IP, DP = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    sig = {
        "stokes_default_params": (None, [ctypes.POINTER(stokes_params)]),
        "stokes_hierarchy_create": (I, [I, D, ctypes.POINTER(stokes_params), VP, ctypes.POINTER(P)]),
        "stokes_hierarchy_destroy": (I, [P]),
        "stokes_level_info": (I, [P, IP, IP]),
        "stokes_level_n": (I, [P, I, IP]),
        "stokes_level_tile": (I, [P, I, IP]),
        "stokes_assemble_rhs": (I, [P, VP, VP, VP]),
        "stokes_apply_operator": (I, [P, I, VP, VP]),
        "stokes_residual": (I, [P, I, VP, VP, VP]),
        "stokes_vanka_sweep": (I, [P, I, VP, VP, VP]),
        "stokes_relaxation_sweep": (I, [P, I, VP, VP, VP]),
        "stokes_device_status": (I, [P]),
        "stokes_test_set_wait_limit": (I, [P, I]),
        "stokes_test_set_alloc_limit": (None, [ctypes.c_longlong]),
        "stokes_test_set_grid_barrier": (I, [P, I, I]),
        "stokes_tail_info": (I, [P, IP, IP, IP]),
        "stokes_restrict": (I, [P, I, VP, VP]),
        "stokes_prolong_add": (I, [P, I, VP, VP]),
        "stokes_coarse_solve": (I, [P, VP, VP]),
        "stokes_initial_guess": (I, [P, VP, VP]),
        "stokes_vcycle_apply": (I, [P, VP, VP]),
        "stokes_fgmres_solve": (I, [P, VP, VP, IP, DP]),
        "stokes_solve_adjoint": (I, [P, VP, VP, VP, IP, DP]),
        "stokes_rhs_transpose": (I, [P, VP, VP]),
        "stokes_batched_solve": (I, [ctypes.POINTER(P), I, ctypes.POINTER(VP), ctypes.POINTER(VP), IP, DP]),
        "stokes_measure_fp64_peak": (I, [VP, DP]),
        "stokes_stats_enable_timing": (I, [P, I]),
        "stokes_stats_reset": (I, [P]),
        "stokes_stats_read": (I, [P, ctypes.POINTER(stokes_stats)]),
        "stokes_residual_norm_noalloc": (I, [I, D, VP, VP, VP, VP]),
        "stokes_batch_create": (I, [I, IP, D, ctypes.POINTER(stokes_params), VP, ctypes.POINTER(P)]),
        "stokes_batch_destroy": (I, [P]),
        "stokes_batch_hierarchy": (I, [P, I, ctypes.POINTER(P)]),
        "stokes_batch_solve": (I, [P, ctypes.POINTER(VP), ctypes.POINTER(VP), IP, DP]),
        "stokes_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    """Names of the C entry points the binding declares (all must resolve in the library)."""
    return ["stokes_default_params", "stokes_hierarchy_create", "stokes_hierarchy_destroy",
            "stokes_level_info", "stokes_level_n", "stokes_level_tile", "stokes_assemble_rhs",
            "stokes_apply_operator",
            "stokes_residual", "stokes_vanka_sweep", "stokes_relaxation_sweep", "stokes_device_status",
            "stokes_test_set_wait_limit", "stokes_test_set_alloc_limit", "stokes_test_set_grid_barrier",
            "stokes_tail_info", "stokes_restrict", "stokes_prolong_add",
            "stokes_coarse_solve", "stokes_initial_guess", "stokes_vcycle_apply", "stokes_fgmres_solve",
            "stokes_solve_adjoint", "stokes_rhs_transpose", "stokes_batched_solve",
            "stokes_measure_fp64_peak", "stokes_stats_enable_timing", "stokes_stats_reset", "stokes_stats_read",
            "stokes_residual_norm_noalloc", "stokes_batch_create", "stokes_batch_destroy",
            "stokes_batch_hierarchy", "stokes_batch_solve", "stokes_last_error"]


def _check(st: int, allow=()) -> int:
    if st != STOKES_OK and st not in allow:
        msg = _load().stokes_last_error()
        raise StokesError(st, msg.decode() if msg else "")
    return st


def _ptr(t, n=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


def vec_len(n: int) -> int:
    return 2 * (2 * n + 1) ** 2 + (n + 1) ** 2


def default_params() -> stokes_params:
    p = stokes_params()
    _load().stokes_default_params(ctypes.byref(p))
    return p


# ---- entry points, same names as the C ABI ----

def stokes_hierarchy_create(n: int, viscosity: float = 1.0, params: stokes_params | None = None,
                            stream: torch.cuda.Stream | None = None):
    lib = _load()
    if params is None:
        params = default_params()
    s = (stream or torch.cuda.current_stream()).cuda_stream
    out = ctypes.c_void_p()
    _check(lib.stokes_hierarchy_create(int(n), float(viscosity), ctypes.byref(params),
                                       ctypes.c_void_p(s), ctypes.byref(out)))
    return out


def stokes_hierarchy_destroy(h) -> None:
    _check(_load().stokes_hierarchy_destroy(h))


def stokes_level_info(h) -> tuple[int, int]:
    L, n = ctypes.c_int(), ctypes.c_int()
    _check(_load().stokes_level_info(h, ctypes.byref(L), ctypes.byref(n)))
    return L.value, n.value


def stokes_level_n(h, level: int) -> int:
    v = ctypes.c_int()
    _check(_load().stokes_level_n(h, int(level), ctypes.byref(v)))
    return v.value


def stokes_level_tile(h, level: int) -> int:
    v = ctypes.c_int()
    _check(_load().stokes_level_tile(h, int(level), ctypes.byref(v)))
    return v.value


def stokes_assemble_rhs(h, f_nodal, u_dirichlet, b, n: int) -> None:
    nq = 2 * n + 1
    _check(_load().stokes_assemble_rhs(h, _ptr(f_nodal, 2 * nq * nq, "f_nodal"),
                                       _ptr(u_dirichlet, 2 * nq * nq, "u_dirichlet"),
                                       _ptr(b, vec_len(n), "b")))


def stokes_apply_operator(h, level: int, x, y) -> None:
    N = vec_len(stokes_level_n(h, level))
    _check(_load().stokes_apply_operator(h, int(level), _ptr(x, N, "x"), _ptr(y, N, "y")))


def stokes_residual(h, level: int, b, x, r) -> None:
    N = vec_len(stokes_level_n(h, level))
    _check(_load().stokes_residual(h, int(level), _ptr(b, N, "b"), _ptr(x, N, "x"), _ptr(r, N, "r")))


def stokes_vanka_sweep(h, level: int, x, b, x_out) -> None:
    N = vec_len(stokes_level_n(h, level))
    _check(_load().stokes_vanka_sweep(h, int(level), _ptr(x, N, "x"), _ptr(b, N, "b"),
                                      _ptr(x_out, N, "x_out")))


def stokes_relaxation_sweep(h, level: int, x, b, x_out) -> None:
    N = vec_len(stokes_level_n(h, level))
    _check(_load().stokes_relaxation_sweep(h, int(level), _ptr(x, N, "x"), _ptr(b, N, "b"),
                                           _ptr(x_out, N, "x_out")))


def stokes_device_status(h, allow_timeout: bool = False) -> int:
    return _check(_load().stokes_device_status(h), allow=(STOKES_ERR_TIMEOUT,) if allow_timeout else ())


def stokes_test_set_wait_limit(h, polls: int) -> None:
    _check(_load().stokes_test_set_wait_limit(h, int(polls)))


def stokes_test_set_alloc_limit(nbytes: int) -> None:
    _load().stokes_test_set_alloc_limit(int(nbytes))


def stokes_test_set_grid_barrier(h, polls: int, withhold_cta: int = -1) -> None:
    _check(_load().stokes_test_set_grid_barrier(h, int(polls), int(withhold_cta)))


def stokes_tail_info(h) -> tuple[int, int, int]:
    t, s, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_load().stokes_tail_info(h, ctypes.byref(t), ctypes.byref(s), ctypes.byref(c)))
    return t.value, s.value, c.value


def stokes_restrict(h, level: int, r_fine, r_coarse) -> None:
    Nf = vec_len(stokes_level_n(h, level))
    Nc = vec_len(stokes_level_n(h, level - 1))
    _check(_load().stokes_restrict(h, int(level), _ptr(r_fine, Nf, "r_fine"), _ptr(r_coarse, Nc, "r_coarse")))


def stokes_prolong_add(h, level: int, e_coarse, x_fine) -> None:
    Nf = vec_len(stokes_level_n(h, level))
    Nc = vec_len(stokes_level_n(h, level - 1))
    _check(_load().stokes_prolong_add(h, int(level), _ptr(e_coarse, Nc, "e_coarse"), _ptr(x_fine, Nf, "x_fine")))


def stokes_coarse_solve(h, r, e) -> None:
    N = vec_len(stokes_level_n(h, 0))
    _check(_load().stokes_coarse_solve(h, _ptr(r, N, "r"), _ptr(e, N, "e")))


def stokes_initial_guess(h, b, x0) -> None:
    _, n = stokes_level_info(h)
    N = vec_len(n)
    _check(_load().stokes_initial_guess(h, _ptr(b, N, "b"), _ptr(x0, N, "x0")))


def stokes_vcycle_apply(h, r, z) -> None:
    _, n = stokes_level_info(h)
    N = vec_len(n)
    _check(_load().stokes_vcycle_apply(h, _ptr(r, N, "r"), _ptr(z, N, "z")))


def stokes_fgmres_solve(h, b, x, allow_not_converged: bool = False) -> tuple[int, float, int]:
    _, n = stokes_level_info(h)
    N = vec_len(n)
    it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
    st = _check(_load().stokes_fgmres_solve(h, _ptr(b, N, "b"), _ptr(x, N, "x"), ctypes.byref(it),
                                            ctypes.byref(rel)),
                allow=(STOKES_NOT_CONVERGED,) if allow_not_converged else ())
    return it.value, rel.value, st


def stokes_solve_adjoint(h, g, lam, grad_f=None) -> tuple[int, float]:
    _, n = stokes_level_info(h)
    N = vec_len(n)
    nq = 2 * n + 1
    it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
    _check(_load().stokes_solve_adjoint(h, _ptr(g, N, "g"), _ptr(lam, N, "lambda"),
                                        _ptr(grad_f, 2 * nq * nq, "grad_f"), ctypes.byref(it),
                                        ctypes.byref(rel)))
    return it.value, rel.value


def stokes_rhs_transpose(h, lam, grad_f) -> None:
    _, n = stokes_level_info(h)
    nq = 2 * n + 1
    _check(_load().stokes_rhs_transpose(h, _ptr(lam, vec_len(n), "lambda"), _ptr(grad_f, 2 * nq * nq, "grad_f")))


def stokes_batched_solve(hs, bs, xs) -> tuple[list[int], list[float]]:
    k = len(hs)
    H = (ctypes.c_void_p * k)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in hs])
    B = (ctypes.c_void_p * k)(*[b.data_ptr() for b in bs])
    X = (ctypes.c_void_p * k)(*[x.data_ptr() for x in xs])
    for h, b, x in zip(hs, bs, xs):
        N = vec_len(stokes_level_info(h)[1])
        _ptr(b, N, "b")
        _ptr(x, N, "x")
    it = (ctypes.c_int * k)()
    rel = (ctypes.c_double * k)()
    _check(_load().stokes_batched_solve(H, k, B, X, it, rel))
    return list(it), list(rel)


def stokes_measure_fp64_peak(stream: torch.cuda.Stream | None = None) -> float:
    """FP64 FMA throughput of the current device in GFLOP/s (measured; synchronises)."""
    s = (stream or torch.cuda.current_stream()).cuda_stream
    g = ctypes.c_double(0.0)
    _check(_load().stokes_measure_fp64_peak(ctypes.c_void_p(s), ctypes.byref(g)))
    return g.value


def stokes_stats_enable_timing(h, enable: bool) -> None:
    _check(_load().stokes_stats_enable_timing(h, int(bool(enable))))


def stokes_stats_reset(h) -> None:
    _check(_load().stokes_stats_reset(h))


def stokes_stats_read(h) -> dict:
    st = stokes_stats()
    _check(_load().stokes_stats_read(h, ctypes.byref(st)))
    return {"kernel_launches": st.kernel_launches, "vcycles": st.vcycles,
            "sweeps_timed": st.sweeps_timed, "sweep_ms": st.sweep_ms, "tc_launches": st.tc_launches}


def stokes_residual_norm_noalloc(n: int, viscosity: float, b, x, norm,
                                 stream: torch.cuda.Stream | None = None) -> None:
    """||b - A x|| into the one-element device tensor `norm`; allocates nothing (see the header)."""
    N = vec_len(n)
    s = (stream or torch.cuda.current_stream()).cuda_stream
    _check(_load().stokes_residual_norm_noalloc(int(n), float(viscosity), _ptr(b, N, "b"), _ptr(x, N, "x"),
                                                _ptr(norm, 1, "norm"), ctypes.c_void_p(s)))


def stokes_batch_create(ns, viscosity: float = 1.0, params: stokes_params | None = None,
                        stream: torch.cuda.Stream | None = None):
    lib = _load()
    if params is None:
        params = default_params()
    s = (stream or torch.cuda.current_stream()).cuda_stream
    arr = (ctypes.c_int * len(ns))(*[int(v) for v in ns])
    out = ctypes.c_void_p()
    _check(lib.stokes_batch_create(len(ns), arr, float(viscosity), ctypes.byref(params), ctypes.c_void_p(s),
                                   ctypes.byref(out)))
    return out


def stokes_batch_destroy(bh) -> None:
    _check(_load().stokes_batch_destroy(bh))


def stokes_batch_hierarchy(bh, k: int):
    out = ctypes.c_void_p()
    _check(_load().stokes_batch_hierarchy(bh, int(k), ctypes.byref(out)))
    return out


def stokes_batch_solve(bh, rhs, xs, allow_not_converged: bool = False):
    k = len(rhs)
    for i, (b, x) in enumerate(zip(rhs, xs)):
        h = stokes_batch_hierarchy(bh, i)
        N = vec_len(stokes_level_info(h)[1])
        _ptr(b, N, "rhs")
        _ptr(x, N, "x")
    B = (ctypes.c_void_p * k)(*[b.data_ptr() for b in rhs])
    X = (ctypes.c_void_p * k)(*[x.data_ptr() for x in xs])
    it = (ctypes.c_int * k)()
    rel = (ctypes.c_double * k)()
    st = _check(_load().stokes_batch_solve(bh, B, X, it, rel),
                allow=(STOKES_NOT_CONVERGED,) if allow_not_converged else ())
    return list(it), list(rel), st


class Batch:
    """Owns a stokes_batch: independent problems (sizes may differ) solved in lockstep."""

    def __init__(self, ns, viscosity: float = 1.0, **kw):
        p = default_params()
        for key, val in kw.items():
            setattr(p, key, val)
        self.ns = list(ns)
        self.handle = stokes_batch_create(self.ns, viscosity, p)

    def hierarchy(self, k: int):
        return stokes_batch_hierarchy(self.handle, k)

    def assemble_rhs(self, k: int, f_nodal, u_dirichlet):
        # problem k runs on a stream of its own: order it after torch's work and back
        n = self.ns[k]
        b = torch.empty(vec_len(n), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        stokes_assemble_rhs(self.hierarchy(k), f_nodal, u_dirichlet, b, n)
        torch.cuda.synchronize()
        return b

    def solve(self, rhs, allow_not_converged: bool = False):
        xs = []
        for k, b in enumerate(rhs):
            x = torch.empty_like(b)
            stokes_initial_guess(self.hierarchy(k), b, x)
            xs.append(x)
        torch.cuda.synchronize()
        it, rel, st = stokes_batch_solve(self.handle, rhs, xs, allow_not_converged)
        return xs, it, rel

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            stokes_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stokes_last_error() -> str:
    m = _load().stokes_last_error()
    return m.decode() if m else ""


# ---- convenience wrapper ----

@dataclass
class Hierarchy:
    """Owns a stokes_hierarchy handle; destroys it on close()/garbage collection."""

    n: int
    viscosity: float = 1.0
    nu1: int = 2
    nu2: int = 2
    omega: float = 0.7
    coarse_n: int = 4
    restart: int = 30
    maxit: int = 1000
    rtol: float = 1e-8
    prec: int = STOKES_FP64
    tile: int = -1
    smoother: int = STOKES_SMOOTHER_SHARED
    bs_t: float = 1.0
    bs_omega: float = 1.0
    bs_jacobi_weight: float = 1.0
    bs_jacobi_iters: int = 2
    cycle: int = 1
    precond: int = 0
    bt_cycles: int = 3
    bt_nu: int = 3
    bt_omega_u: float = 1.0
    bt_omega_p: float = 0.6
    tail_n: int = 0
    orth: int = 0

    def __post_init__(self):
        p = default_params()
        p.nu1, p.nu2, p.omega, p.coarse_n = self.nu1, self.nu2, self.omega, self.coarse_n
        p.restart, p.maxit, p.rtol, p.prec = self.restart, self.maxit, self.rtol, self.prec
        p.tile = self.tile
        p.smoother = self.smoother
        p.bs_t, p.bs_omega = self.bs_t, self.bs_omega
        p.bs_jacobi_weight, p.bs_jacobi_iters = self.bs_jacobi_weight, self.bs_jacobi_iters
        p.cycle = self.cycle
        p.precond, p.bt_cycles, p.bt_nu = self.precond, self.bt_cycles, self.bt_nu
        p.bt_omega_u, p.bt_omega_p = self.bt_omega_u, self.bt_omega_p
        p.tail_n = self.tail_n
        p.orth = self.orth
        self.handle = stokes_hierarchy_create(self.n, self.viscosity, p)
        self.levels, _ = stokes_level_info(self.handle)
        self.N = vec_len(self.n)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            stokes_hierarchy_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_n(self, level: int) -> int:
        return stokes_level_n(self.handle, level)

    def empty(self, level: int | None = None) -> torch.Tensor:
        n = self.n if level is None else self.level_n(level)
        return torch.empty(vec_len(n), dtype=torch.float64, device="cuda")

    def assemble_rhs(self, f_nodal, u_dirichlet):
        b = self.empty()
        stokes_assemble_rhs(self.handle, f_nodal, u_dirichlet, b, self.n)
        return b

    def apply(self, x, level=None):
        level = self.levels - 1 if level is None else level
        y = torch.empty_like(x)
        stokes_apply_operator(self.handle, level, x, y)
        return y

    def residual(self, b, x, level=None):
        level = self.levels - 1 if level is None else level
        r = torch.empty_like(b)
        stokes_residual(self.handle, level, b, x, r)
        return r

    def sweep(self, x, b, level=None):
        level = self.levels - 1 if level is None else level
        out = torch.empty_like(b)
        stokes_vanka_sweep(self.handle, level, x, b, out)
        return out

    def relax(self, x, b, level=None):
        """One sweep of the V-cycle's smoother in the hierarchy's arithmetic (x None: zero guess)."""
        level = self.levels - 1 if level is None else level
        out = torch.empty_like(b)
        stokes_relaxation_sweep(self.handle, level, x, b, out)
        return out

    def vcycle(self, r):
        z = torch.empty_like(r)
        stokes_vcycle_apply(self.handle, r, z)
        return z

    def solve(self, b, x0=None, allow_not_converged=False):
        if x0 is None:
            x = torch.empty_like(b)
            stokes_initial_guess(self.handle, b, x)
        else:
            x = x0.clone()
        it, rel, st = stokes_fgmres_solve(self.handle, b, x, allow_not_converged)
        return x, it, rel

    def adjoint(self, g):
        lam = torch.empty_like(g)
        grad = torch.empty(2 * (2 * self.n + 1) ** 2, dtype=torch.float64, device=g.device)
        it, rel = stokes_solve_adjoint(self.handle, g, lam, grad)
        return lam, grad, it, rel
