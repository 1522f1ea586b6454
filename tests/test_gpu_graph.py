"""A V-cycle captured as a CUDA graph and replayed equals the eager V-cycle bit for bit.

Capture exercises what eager runs do not: the programmatic-dependent launches
of every kernel as graph edges, and the BF16 form's fork of the boundary ring
onto the hierarchy's second stream and its join, under stream capture.  Every
kernel sums in a fixed order (no atomics), so the results must be identical.
"""
import numpy as np
import pytest
import torch

import stokes_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2401_06277_gb300 as p
    from paper_2401_06277_gb300 import build
    build.build()
    return p


@pytest.mark.parametrize("prec,smoother,tail_n,tile", [(0, 0, 0, -1), (1, 0, 0, -1), (2, 0, 0, -1), (1, 2, 0, -1),
                                                       (0, 1, 0, -1), (1, 0, 128, -1), (2, 0, 128, -1),
                                                       (1, 0, 0, 3), (2, 0, 0, 3)])
@pytest.mark.parametrize("n", [16, 64, 128])
def test_graph_replay_equals_eager_vcycle(pkg, n, prec, smoother, tail_n, tile):
    """tail_n = 128: the coarse levels as the persistent cooperative launch, captured too;
    tile = 3 in the mixed forms: the strip sweeps (with their ring fork) wherever they fit."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        H = pkg.Hierarchy(n, prec=prec, smoother=smoother, tail_n=tail_n, tile=tile)
        b = torch.from_numpy(si.random_vector(n, 31)).cuda()
        z_eager = torch.empty_like(b)
        z_graph = torch.full_like(b, float("nan"))
        pkg.stokes_vcycle_apply(H.handle, b, z_eager)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            pkg.stokes_vcycle_apply(H.handle, b, z_graph)
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        a, c = z_eager.cpu().numpy(), z_graph.cpu().numpy()
        del g
        H.close()
    torch.cuda.current_stream().wait_stream(s)
    assert np.isfinite(a).all()
    assert np.array_equal(a, c), float(np.abs(a - c).max())
