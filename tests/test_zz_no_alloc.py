"""swe_rhs_p1_noalloc -- the allocation-free right-hand side -- against the
context path swe_rhs on the same inputs, through the C ABI (needs a GB300).

The entry point serves callers that cannot allocate device memory (an
application that hands the solver fixed, pre-allocated buffers and forbids
cudaMalloc/cudaFree, for instance because its device memory is partitioned
up front or because an allocation would synchronise its pipelined streams).
Its intermediate values live in one fixed device array that every call
shares, so two calls in a row with different inputs must each match the
context path, and the FP64 oracle (the paper's Sect. 2-3 scheme for p = 1
with land walls) to 1e-12 of the largest entry.  Invalid mesh data (a vertex
id out of range, a clockwise triangle, neighbour entries that are out of range
or one-sided) must give NaN rows or land edges, never an access outside the
caller's arrays: each case is compared with the oracle on the mesh that the
documented reading describes.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also
passes alone.
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
    P = O.Params(g=9.81)
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
        r_o = m.rhs(P, c)
        assert np.all(r_o[:, 3:, :] == 0.0)
        assert np.abs(got - r_o[:, :3, :]).max() <= 1e-12 * np.abs(r_o).max()
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


def _noalloc(xy, hv, tri, nbr, c3, g=9.81):
    import torch
    dev = torch.device("cuda")
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(dev)  # noqa: E731
    out = torch.full((3, 3, len(tri)), float("nan"), dtype=torch.float64, device=dev)
    swedg.rhs_p1_noalloc(t(xy, np.float64), t(hv, np.float64), t(tri, np.int32), t(nbr, np.int32),
                         t(c3, np.float64), g, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _case(n=16, seed=9):
    L = 1e4
    xy, tri = inputs.split_square_mesh(n, L, jitter=0.2, seed=seed)
    hv = inputs.fourier_bathymetry(xy, L, lo=20.0, hi=200.0, seed=seed + 1)
    ic = lambda x, y: (0.3 * np.exp(-((x - 5e3) ** 2 + (y - 6e3) ** 2) / 5e6), 1.5 + 0.0 * x, -0.5 + 0.0 * y)  # noqa: E731
    c = O.Mesh(xy, tri, hv, np.ones(len(tri), np.int8)).project_state(ic)
    return xy, tri, hv, c


def _close(a, b):
    return np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_noalloc_unusable_elements_get_nan_rows_and_are_land_to_their_neighbours():
    """An element with a vertex id outside [0, nv), and a clockwise element:
    NaN rows for that element; every other element equals the oracle on the
    mesh without it (its neighbours see a land edge there)."""
    build.build()
    swedg.load()
    xy, tri, hv, c = _case()
    nbr = neighbours(tri)
    ne, nv = len(tri), len(xy)
    P = O.Params(g=9.81)
    for kind, e_bad in (("vertex id", 37), ("clockwise", 200)):
        tri_b = tri.copy()
        if kind == "vertex id":
            tri_b[e_bad, 1] = nv  # one past the last vertex
        else:
            tri_b[e_bad, [1, 2]] = tri_b[e_bad, [2, 1]]
        got = _noalloc(xy, hv, tri_b, nbr, c[:, :3])
        assert np.all(np.isnan(got[:, :, e_bad])), kind
        keep = np.arange(ne) != e_bad
        assert np.all(np.isfinite(got[:, :, keep])), kind
        m = O.Mesh(xy, tri[keep], hv, np.ones(ne - 1, np.int8))
        ref = m.rhs(P, c[:, :, keep])[:, :3]
        assert _close(got[:, :, keep], ref), kind


def test_noalloc_neighbour_entries_out_of_range_or_one_sided_are_land():
    """The interior edges along one grid line are cut in the neighbour map:
    on the west side their entries point outside [0, ne), on the east side
    they still name the west element (one-sided).  Both sides must then see a
    land wall there: the oracle computes the same mesh with the line's
    vertices duplicated for the east side (two domains with a wall between)."""
    build.build()
    swedg.load()
    n = 16
    xy, tri, hv, c = _case(n=n)
    nbr = neighbours(tri)
    ne, nv = len(tri), len(xy)
    col = lambda v: v // (n + 1)  # noqa: E731  vertex column index of the split-square grid
    cut = n // 2
    east = np.array([col(tri[e]).min() >= cut for e in range(ne)])
    west = ~east
    nbr_b = nbr.copy()
    cut_edges = 0
    for e in np.nonzero(west)[0]:
        for k in range(3):
            if nbr[e, k] >= 0 and east[nbr[e, k]]:
                nbr_b[e, k] = ne + 5 + k  # out of range on the west side
                cut_edges += 1
    assert cut_edges == n
    got = _noalloc(xy, hv, tri, nbr_b, c[:, :3])
    assert np.all(np.isfinite(got))
    # the oracle's mesh: vertices on the cut line duplicated for the east elements
    line = np.nonzero(col(np.arange(nv)) == cut)[0]
    dup = {int(v): nv + i for i, v in enumerate(line)}
    xy2 = np.concatenate([xy, xy[line]])
    hv2 = np.concatenate([hv, hv[line]])
    tri2 = tri.copy()
    for e in np.nonzero(east)[0]:
        tri2[e] = [dup.get(int(v), int(v)) for v in tri[e]]
    m = O.Mesh(xy2, tri2, hv2, np.ones(ne, np.int8))
    assert int((m.neighbours()["nb"] < 0).sum()) == int((neighbours(tri) < 0).sum()) + 2 * n
    ref = m.rhs(O.Params(g=9.81), c)[:, :3]
    assert _close(got, ref)
    # and the intact map still gives the uncut oracle
    ref_full = O.Mesh(xy, tri, hv, np.ones(ne, np.int8)).rhs(O.Params(g=9.81), c)[:, :3]
    assert _close(_noalloc(xy, hv, tri, nbr, c[:, :3]), ref_full)
    assert not _close(got, ref_full)


def test_noalloc_rejects_a_non_positive_or_non_finite_g():
    build.build()
    swedg.load()
    xy, tri, hv, c = _case(n=4)
    for g in (0.0, -9.81, float("nan"), float("inf")):
        with pytest.raises(swedg.SweError) as ei:
            _noalloc(xy, hv, tri, neighbours(tri), c[:, :3], g=g)
        assert ei.value.code == -1
