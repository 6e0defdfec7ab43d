"""Pins of the oracle's basis and reference tensors (no GPU).

The oracle integrates monomial expansions exactly; here every tensor is
re-derived by Gauss quadrature of an independent scipy evaluation of the
Dubiner basis, and tied together by integration-by-parts identities and the
orthogonality zeros.  Cited: Sect. 2 (hierarchical orthonormal basis, K(p)),
Eq. (13) (integrals of basis products), Sect. 3 (truncated system).
"""
import os

import numpy as np
import pytest

import dgref
import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def err(a, b):
    """max abs difference relative to the largest entry (entries reach ~45);
    the scipy quadrature reference itself is good to ~1e-14 relative"""
    return np.abs(a - b).max() / max(1.0, np.abs(b).max())


@pytest.fixture(scope="module")
def T():
    return O.tensors()


@pytest.fixture(scope="module")
def quad():
    x, y, w = dgref.tri_rule(16)
    v, vx, vy = dgref.basis(x, y)
    return x, y, w, v, vx, vy


def test_golden_K_of_p():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "paper_K.txt")) if l.strip() and l[0] != "#"]
    for p, K in rows:
        assert O.K_OF_P[int(p)] == int(K)
        assert (int(p) + 1) * (int(p) + 2) // 2 == int(K)
    deg = O.degrees()
    for p in range(5):
        assert np.sum(deg <= p) == O.K_OF_P[p]


def test_golden_truncation_cases():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "paper_Ktr.txt")) if l.strip() and l[0] != "#"]
    for p, i, j, K in rows:
        assert O.Ktr(int(i) - 1, int(j) - 1) == int(K), (p, i, j)


def test_basis_matches_independent_formula():
    rng = np.random.default_rng(0)
    a = rng.uniform(0, 1, 200); b = rng.uniform(0, 1, 200)
    x = a * (1 - b); y = b
    ref, _, _ = dgref.basis(x, y)
    C = O.basis_monomials()
    pd = C.shape[1]
    val = np.zeros_like(ref)
    for ia in range(pd):
        for ib in range(pd - ia):
            val += C[:, ia, ib, None] * x ** ia * y ** ib
    assert np.abs(val - ref).max() < 1e-12


def test_orthonormal(T, quad):
    x, y, w, v, vx, vy = quad
    M = (v * w) @ v.T
    assert np.abs(M - np.eye(15)).max() < 1e-13
    assert np.abs(T["M"] - np.eye(15)).max() < 1e-14
    assert abs(v[0, 0] - np.sqrt(2.0)) < 1e-15


def test_volume_tensors_by_quadrature(T, quad):
    x, y, w, v, vx, vy = quad
    dv = (vx, vy)
    for k in range(2):
        D = np.einsum("n,qn,in->qi", w, dv[k], v)
        assert err(D, T["D"][k]) < 1e-14
        G = np.einsum("n,qn,in,jn->qij", w, dv[k], v, v)
        assert err(G, T["G"][k]) < 1e-14
    Tq = np.einsum("n,an,in,jn->aij", w, v, v, v)
    assert err(Tq, T["T"]) < 1e-14
    lam = np.stack([1 - x - y, x, y])
    L = np.einsum("n,vn,in->vi", w, lam, v)
    assert np.abs(L - T["L"]).max() < 1e-14


def test_edge_tensors_by_quadrature(T):
    s, w = dgref.gauss01(12)
    B = [dgref.basis(*dgref.edge_points(k, s))[0] for k in range(3)]
    Br = [dgref.basis(*dgref.edge_points(k, 1.0 - s))[0] for k in range(3)]
    for k in range(3):
        S2 = np.einsum("g,qg,ig->qi", w, B[k], B[k])
        S3 = np.einsum("g,qg,ig,jg->qij", w, B[k], B[k], B[k])
        assert err(S2, T["S2"][k]) < 1e-14
        assert err(S3, T["S3"][k]) < 1e-14
        for kk in range(3):
            X2 = np.einsum("g,qg,ig->qi", w, B[k], Br[kk])
            X3 = np.einsum("g,qg,ig,jg->qij", w, B[k], Br[kk], Br[kk])
            assert err(X2, T["X2"][k, kk]) < 1e-14
            assert err(X3, T["X3"][k, kk]) < 1e-14


def test_integration_by_parts(T):
    """int phi_i d_k phi_q + int phi_q d_k phi_i = sum_edges |E_hat| n_k int phi_i phi_q
    and the three-index analogue tie the volume tensors to the edge tensors."""
    # reference edge lengths and outward normals (edge k opposite vertex k)
    Lh = np.array([np.sqrt(2.0), 1.0, 1.0])
    nh = np.array([[1.0, 1.0], [-1.0, 0.0], [0.0, -1.0]])
    nh[0] /= np.sqrt(2.0)
    D, G, S2, S3 = T["D"], T["G"], T["S2"], T["S3"]
    for k in range(2):
        lhs = D[k] + D[k].T
        rhs = sum(Lh[e] * nh[e, k] * S2[e] for e in range(3))
        assert err(lhs, rhs) < 2e-15
        lhs3 = G[k] + np.transpose(G[k], (1, 0, 2)) + np.transpose(G[k], (2, 1, 0))
        rhs3 = sum(Lh[e] * nh[e, k] * S3[e] for e in range(3))
        assert err(lhs3, rhs3) < 2e-15


def test_structural_zeros(T):
    deg = O.degrees()
    D, G, Tt = T["D"], T["G"], T["T"]
    for q in range(15):
        for i in range(15):
            if deg[i] >= deg[q]:
                assert np.abs(D[:, q, i]).max() < 1e-15
            for j in range(15):
                dq, di, dj = deg[q], deg[i], deg[j]
                if dq == 0 or di > dj + dq - 1 or dj > di + dq - 1 or (dq == 1 and i != j):
                    assert np.abs(G[:, q, i, j]).max() < 1e-15
                if dq > di + dj or di > dq + dj or dj > dq + di:
                    assert abs(Tt[q, i, j]) < 1e-15
    # T is symmetric in all three indices, G in its last two
    assert np.abs(Tt - np.transpose(Tt, (1, 0, 2))).max() < 1e-15
    assert np.abs(Tt - np.transpose(Tt, (2, 1, 0))).max() < 1e-15
    assert np.abs(G - np.transpose(G, (0, 1, 3, 2))).max() < 1e-15


def test_truncation_rule():
    deg = O.degrees()
    for i in range(15):
        for j in range(15):
            assert O.Ktr(i, j) == O.K_OF_P[max(deg[i], deg[j])]


def test_tri_rule_is_exact():
    x, y, w = O.tri_rule(6)
    import math
    for a in range(8):
        for b in range(10 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.sum(w * x ** a * y ** b) - exact) < 1e-15
