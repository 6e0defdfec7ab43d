"""The C ABI library builds, loads and exports every declared symbol; its own
reference tables agree with the oracle's (host-only calls, no GPU)."""
import math
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2311_11348_gb300 import build, swedg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return swedg.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "swedg.h")).read()
    return sorted(set(re.findall(r"\b(swe_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_binding_symbols():
    assert sorted(swedg.SYMBOLS) == declared_symbols()


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_library_tensors_match_oracle(lib):
    D, G, T = swedg.reference_tensors()
    t = O.tensors()
    for a, b in ((D, t["D"]), (G, t["G"]), (T, t["T"])):
        assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()


def test_p1_mass_tensor_structure_the_velocity_solve_uses(lib):
    """the P1 velocity solve drops T[0][i][j] = T[i][0][j] = phihat_1 delta_ij
    (orthonormal basis, constant phihat_1 = sqrt 2) from its arithmetic"""
    _, _, T = swedg.reference_tensors()
    for i in range(3):
        for j in range(3):
            assert abs(T[0, i, j] - math.sqrt(2.0) * (i == j)) < 1e-14
            assert abs(T[i, 0, j] - math.sqrt(2.0) * (i == j)) < 1e-14


@pytest.mark.parametrize("npts,pmax", [(2, 1), (4, 2), (5, 3), (7, 4)])
def test_factored_edge_tables_reproduce_edge_tensors(lib, npts, pmax):
    """The library applies the edge tensors of the quadrature-free scheme in
    factored form: S3 = sum_g w_g B B B, X3 with the neighbour traversed
    backwards.  Exact for the polynomial degrees of that max order."""
    s, w, B = swedg.edge_table(npts)
    t = O.tensors()
    K = (pmax + 1) * (pmax + 2) // 2
    S3 = np.einsum("g,kqg,kig,kjg->kqij", w, B, B, B)[:, :K, :K, :K]
    X3 = np.einsum("g,kqg,lig,ljg->klqij", w, B, B[:, :, ::-1], B[:, :, ::-1])[..., :K, :K, :K]
    assert np.abs(S3 - t["S3"][:, :K, :K, :K]).max() <= 1e-14 * np.abs(t["S3"]).max()
    assert np.abs(X3 - t["X3"][..., :K, :K, :K]).max() <= 1e-14 * np.abs(t["X3"]).max()
    assert abs(w.sum() - 1.0) < 1e-15


def test_noalloc_wrapper_rejects_bad_arguments_before_the_call():
    """rhs_p1_noalloc hands raw pointers to kernels that read and write fixed
    extents, so the binding refuses anything but contiguous CUDA tensors of the
    right dtype and shape (checked on the host, no GPU needed)"""
    import torch
    nv, ne = 9, 8
    good = dict(xy=torch.zeros((nv, 2), dtype=torch.float64), hv=torch.ones(nv, dtype=torch.float64),
                tri=torch.zeros((ne, 3), dtype=torch.int32), nbr=torch.full((ne, 3), -1, dtype=torch.int32),
                c=torch.zeros((3, 3, ne), dtype=torch.float64), out=torch.zeros((3, 3, ne), dtype=torch.float64))
    bad = {
        "numpy": ("c", np.zeros((3, 3, ne))),
        "dtype": ("c", torch.zeros((3, 3, ne), dtype=torch.float32)),
        "int64 mesh": ("tri", torch.zeros((ne, 3), dtype=torch.int64)),
        "short out": ("out", torch.zeros((3, 3, ne - 1), dtype=torch.float64)),
        "hv length": ("hv", torch.ones(nv + 1, dtype=torch.float64)),
        "nbr shape": ("nbr", torch.full((ne, 2), -1, dtype=torch.int32)),
        "strided": ("c", torch.zeros((3, 3, 2 * ne), dtype=torch.float64)[:, :, ::2]),
        "host": ("out", None),  # every tensor of `good` lives on the host
    }
    for what, (name, val) in bad.items():
        args = dict(good)
        if val is not None:
            args[name] = val
        with pytest.raises(ValueError):
            swedg.rhs_p1_noalloc(args["xy"], args["hv"], args["tri"], args["nbr"], args["c"], 9.81, args["out"])
