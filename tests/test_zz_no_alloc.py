"""swe_rhs_p1_noalloc -- the allocation-free right-hand side -- against the
context path swe_rhs on the same inputs, through the C ABI (needs a GB300).

The entry point serves callers that cannot allocate device memory (an
application that hands the solver fixed, pre-allocated buffers and forbids
cudaMalloc/cudaFree, for instance because its device memory is partitioned
up front or because an allocation would synchronise its pipelined streams).
Its intermediate values live in one fixed device array that every call
shares, so two calls in a row with different inputs must each match the
context path.  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes alone.
"""
import numpy as np
import pytest

import oracle as O
from paper_2311_11348_gb300 import build, inputs, swedg

pytestmark = pytest.mark.gpu


def neighbours(tri):
    """element across the edge opposite vertex k, or -1"""
    ne = len(tri)
    nbr = -np.ones((ne, 3), np.int32)
    seen = {}
    for e in range(ne):
        for k in range(3):
            a, b = tri[e, (k + 1) % 3], tri[e, (k + 2) % 3]
            key = (min(a, b), max(a, b))
            if key in seen:
                f, kf = seen.pop(key)
                nbr[e, k] = f
                nbr[f, kf] = e
            else:
                seen[key] = (e, k)
    return nbr


def test_noalloc_matches_context_rhs_on_two_calls():
    import torch
    build.build()
    swedg.load()
    L = 1e4
    xy, tri = inputs.split_square_mesh(24, L, jitter=0.2, seed=7)
    hv = inputs.fourier_bathymetry(xy, L, lo=20.0, hi=200.0, seed=8)
    ne = len(tri)
    m = O.Mesh(xy, tri, hv, np.ones(ne, np.int8))
    states = [
        m.project_state(lambda x, y: (0.4 * np.exp(-((x - 6e3) ** 2 + (y - 4e3) ** 2) / 4e6), 2.0 + 0.0 * x,
                                      -1.0 + 0.0 * y)),
        m.project_state(lambda x, y: (0.1 * np.sin(x / 1e3), 0.5 * np.cos(y / 2e3), 0.3 * np.sin((x + y) / 3e3))),
    ]
    s = swedg.Solver(g=9.81)
    s.set_mesh(xy, tri)
    s.set_bathymetry(hv)
    dev = torch.device("cuda")
    xy_d = torch.from_numpy(np.ascontiguousarray(xy)).to(dev)
    hv_d = torch.from_numpy(np.ascontiguousarray(hv)).to(dev)
    tri_d = torch.from_numpy(np.ascontiguousarray(tri, dtype=np.int32)).to(dev)
    nbr_d = torch.from_numpy(neighbours(tri)).to(dev)
    out_d = torch.empty((3, 3, ne), dtype=torch.float64, device=dev)
    for c in states:  # two calls in a row, different inputs
        ref = s.rhs(c)[:, :3, :]
        c_d = torch.from_numpy(np.ascontiguousarray(c[:, :3, :])).to(dev)
        out_d.fill_(float("nan"))
        torch.cuda.synchronize()
        swedg.rhs_p1_noalloc(xy_d, hv_d, tri_d, nbr_d, c_d, 9.81, out_d)
        torch.cuda.synchronize()
        got = out_d.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    build.build()
    swedg.load()
    dev = torch.device("cuda")
    n = swedg.NOALLOC_MAX_ELEMENTS + 1
    tri = torch.zeros((n, 3), dtype=torch.int32, device=dev)
    nbr = torch.full((n, 3), -1, dtype=torch.int32, device=dev)
    xy = torch.zeros((3, 2), dtype=torch.float64, device=dev)
    hv = torch.ones(3, dtype=torch.float64, device=dev)
    c = torch.zeros((3, 3, n), dtype=torch.float64, device=dev)
    out = torch.zeros((3, 3, n), dtype=torch.float64, device=dev)
    with pytest.raises(swedg.SweError) as ei:
        swedg.rhs_p1_noalloc(xy, hv, tri, nbr, c, 9.81, out)
    assert ei.value.code == -1
