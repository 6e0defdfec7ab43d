"""The C ABI library builds, loads and exports every declared symbol; its own
reference tables agree with the oracle's (host-only calls, no GPU)."""
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
