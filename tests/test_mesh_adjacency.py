"""The library's mesh adjacency (host code of swe_set_mesh, reached through
the context-free swe_mesh_adjacency: no GPU) against a brute-force pairing of
the triangles' edges, on renumbered meshes with clockwise triangles, and its
rejection of invalid meshes."""
import numpy as np
import pytest

from dgref import brute_force_adjacency
from paper_2311_11348_gb300 import build, inputs, swedg


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    swedg.load()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjacency_equals_brute_force_on_renumbered_meshes(seed):
    rng = np.random.default_rng(seed)
    n = 7 + seed
    xy, tri = inputs.split_square_mesh(n, 1.0, jitter=0.2, seed=seed)
    pv = rng.permutation(len(xy))
    xy = xy[np.argsort(pv)]
    tri = pv[tri][rng.permutation(len(tri))].astype(np.int32)
    flip = rng.uniform(size=len(tri)) < 0.3
    tri[flip] = tri[flip][:, [0, 2, 1]]  # clockwise: the library re-orients them internally
    nbr, nbk = swedg.mesh_adjacency(xy, tri)
    rb, rk = brute_force_adjacency(tri)
    assert np.array_equal(nbr, rb) and np.array_equal(nbk, rk)
    assert (nbr < 0).sum() == 4 * n  # the boundary of the split square
    # the relation is mutual
    e, k = np.nonzero(nbr >= 0)
    assert np.array_equal(nbr[nbr[e, k], nbk[e, k]], e)


def test_invalid_meshes_are_rejected():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0], [0.5, -1.0], [2.0, 0.0]])
    good = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    nbr, nbk = swedg.mesh_adjacency(xy, good)
    # the edge (1, 2) is edge 0 of triangle 0 (opposite vertex 0) and edge 1 of triangle 1
    assert nbr.tolist() == [[1, -1, -1], [-1, 0, -1]] and nbk.tolist() == [[1, -1, -1], [-1, 0, -1]]
    cases = {
        "a third triangle on the edge (1, 2)": (np.array([[0, 1, 2], [1, 3, 2], [1, 2, 4]]), -2, "more than 2"),
        "a repeated vertex": (np.array([[0, 1, 2], [1, 1, 3]]), -2, "degenerate"),
        "a vertex id out of range": (np.array([[0, 1, 2], [1, 3, 6]]), -2, "out of range"),
        "collinear vertices": (np.array([[0, 1, 2], [0, 5, 1]]), -2, "degenerate"),
        "no triangles": (np.zeros((0, 3)), -1, "ne >= 1"),
    }
    for what, (tri, code, text) in cases.items():
        with pytest.raises(swedg.SweError) as ei:
            swedg.mesh_adjacency(xy, np.asarray(tri, np.int32))
        assert ei.value.code == code and text in str(ei.value), (what, ei.value.code, str(ei.value))
