"""stokes_residual_norm_noalloc: ||b - A x|| for callers that cannot allocate device memory.

Some callers cannot let a library call cudaMalloc: their device memory is all
owned by another allocator, or they run while a stream is being captured into
a CUDA graph.  This entry point keeps its scratch in a fixed device array
instead.  The test calls it through the C ABI twice in a row (different
inputs, so a stale scratch value would show) and compares each result with
the norm of the residual produced by the existing stokes_residual entry point.
It sits in its own file, collected last, and passes alone or after the rest.
"""
import ctypes
import gc

import numpy as np
import pytest
import torch

import stokes_inputs as si

pytestmark = pytest.mark.gpu

RTOL = 1e-12   # the tolerance of the sweep / V-cycle parity tests


@pytest.fixture(scope="module")
def stokes():
    from paper_2401_06277_gb300 import build, stokes as s
    build.build()
    return s


@pytest.mark.parametrize("n", [16, 64])
def test_noalloc_residual_norm_matches_existing_entry_point(stokes, n):
    h = stokes.Hierarchy(n, viscosity=1.3)
    lvl = h.levels - 1
    lib = stokes._load()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((10, 20)):
        b = torch.from_numpy(si.random_vector(n, seed)).cuda()
        x = torch.from_numpy(si.random_vector(n, seed + 1)).cuda()
        r = torch.empty_like(b)
        stokes.stokes_residual(h.handle, lvl, b, x, r)
        ref = float(torch.linalg.vector_norm(r))
        if call == 1:
            # no Python garbage collection inside the window: a collected tensor
            # of an earlier test would change torch's counter without our call
            gc.collect()
            gc.disable()
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            alloc0 = torch.cuda.memory_allocated()
        try:
            st = lib.stokes_residual_norm_noalloc(n, 1.3, ctypes.c_void_p(b.data_ptr()),
                                                  ctypes.c_void_p(x.data_ptr()),
                                                  ctypes.c_void_p(out.data_ptr()), stream)
            assert st == stokes.STOKES_OK, lib.stokes_last_error()
            torch.cuda.synchronize()
            if call == 1:
                assert torch.cuda.mem_get_info()[0] == free0
                assert torch.cuda.memory_allocated() == alloc0
        finally:
            gc.enable()
        got = float(out.item())
        assert abs(got - ref) <= RTOL * ref, (call, got, ref)
    h.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(stokes):
    lib = stokes._load()
    big = 2 * 8192
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    st = lib.stokes_residual_norm_noalloc(big, 1.0, p, p, p, None)
    assert st == stokes.STOKES_ERR_ARG
    assert b"8192" in lib.stokes_last_error()
    assert lib.stokes_residual_norm_noalloc(0, 1.0, p, p, p, None) == stokes.STOKES_ERR_ARG


@pytest.mark.parametrize("n", [1, 2, 3])
def test_noalloc_residual_norm_on_the_smallest_grids(stokes, n):
    """n = 1..3, below any hierarchy (n >= 4): nearly every row is near the boundary, where
    the Dirichlet masks decide the stencil.  The norm equals ||b - A x|| with the oracle's
    assembled, Dirichlet-eliminated operator (Section 2.2)."""
    from oracle import stokes_oracle as O
    A = O.stokes_operator(O.Mesh(n), 1.3)[0]
    b, x = si.random_vector(n, 40 + n), si.random_vector(n, 50 + n)
    ref = float(np.linalg.norm(b - A @ x))
    lib = stokes._load()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    bd, xd = torch.from_numpy(b).cuda(), torch.from_numpy(x).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.stokes_residual_norm_noalloc(n, 1.3, ctypes.c_void_p(bd.data_ptr()), ctypes.c_void_p(xd.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), stream)
    assert st == stokes.STOKES_OK, lib.stokes_last_error()
    got = float(out.item())
    assert abs(got - ref) <= RTOL * ref, (got, ref)


def test_noalloc_residual_norm_inside_a_captured_graph(stokes):
    """The call a capturing caller makes: after one call outside capture (which looks up
    the scratch address), a second call recorded into a CUDA graph and replayed gives the
    norm of stokes_residual's residual for the inputs the graph reads at replay."""
    n = 16
    h = stokes.Hierarchy(n, viscosity=1.3)
    b = torch.from_numpy(si.random_vector(n, 60)).cuda()
    x = torch.from_numpy(si.random_vector(n, 61)).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stokes.stokes_residual_norm_noalloc(n, 1.3, b, x, out)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            stokes.stokes_residual_norm_noalloc(n, 1.3, b, x, out, stream=s)
    for seed in (62, 63):   # new inputs in place, then replay
        b.copy_(torch.from_numpy(si.random_vector(n, seed)))
        out.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        r = torch.empty_like(b)
        stokes.stokes_residual(h.handle, h.levels - 1, b, x, r)
        ref = float(torch.linalg.vector_norm(r))
        assert abs(float(out.item()) - ref) <= RTOL * ref
    del g
    h.close()
