"""Host-side checks of the tensor-core volume contraction (precision mode
SWE_PREC_MIXED_TF32), no GPU: the library's constant operand images decode,
by the layout the header documents, to the oracle's G tensors of Eq. (13),
split into two TF32 parts; and the GEMM decomposition the
kernel uses (symmetrised coefficient products against those images)
reproduces the direct volume contraction of the momentum rows."""
import numpy as np
import pytest

import oracle as O
from paper_2311_11348_gb300 import build, swedg

DEG = [0, 1, 1, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4]


@pytest.fixture(scope="module")
def lib():
    build.build()
    return swedg.load()


def pairs(K):
    return [(i, j) for j in range(K) for i in range(j + 1)]  # pair index j(j+1)/2 + i


def decode(K, img):
    P = K * (K + 1) // 2
    RS = -(-2 * P // 32) * 32
    RP = -(-P // 32) * 32

    def op(base, R, C):
        out = np.zeros((R, C), np.float32)
        for r in range(R):
            for c in range(C):
                out[r, c] = img[base + (c // 32) * 32 * R + (r // 8) * 256 + ((c % 32) // 4) * 32 + (r % 8) * 4 + c % 4]
        return out

    S = [op(k * 16 * RS, 16, RS) for k in range(2)]
    Pp = [op(32 * RS + k * 32 * RP, 32, RP) for k in range(2)]
    assert len(img) == 32 * RS + 64 * RP
    return P, S, Pp


def used(q, i, j):
    """structurally nonzero and not a base triple (the FP64 base owns q, i, j < 3)"""
    dq, di, dj = DEG[q], DEG[i], DEG[j]
    if q < 3 and i < 3 and j < 3:
        return False
    if dq == 0:
        return False
    if dq == 1:
        return i == j
    return di <= dj + dq - 1 and dj <= di + dq - 1


@pytest.mark.parametrize("K", [6, 10, 15])
def test_operand_images_hold_G_split_into_tf32_head_and_tail(lib, K):
    img = swedg.tc_operand_image(K)
    P, Sp, Pp = decode(K, img)
    G = O.tensors()["G"]
    for a in Sp + Pp:  # every part is a TF32 value: no bits below the 10-bit mantissa
        assert np.all(a.view(np.uint32) & 0x1FFF == 0)
    S = sum(a.astype(np.float64) for a in Sp)
    Pm = sum(a.astype(np.float64) for a in Pp)
    sh = Sp[0]
    floor = 1e-14 * np.abs(G).max()  # the library's tables agree with the oracle's to this
    for k in range(2):
        for q in range(16):
            for pr, (i, j) in enumerate(pairs(K)):
                want = G[k, q, i, j] if (q < K and used(q, i, j)) else 0.0
                tol = 2.0 ** -21 * abs(want) + floor  # the parts sum to G within 2^-22 |G|
                assert abs(S[q, k * P + pr] - want) <= tol, (k, q, i, j)
                assert abs(Pm[16 * k + q, pr] - want) <= tol, (k, q, i, j)
                # part 0 is G rounded to 10 mantissa bits
                if want:
                    assert abs(sh[q, k * P + pr] - want) <= 2.0 ** -11 * abs(want) + floor
    # padding columns and unused rows are exact zeros
    assert not np.any(S[:, 2 * P:]) and not np.any(Pm[:, P:])
    assert not np.any(S[K:]) and not np.any(Pm[K:16]) and not np.any(Pm[16 + K:])


@pytest.mark.parametrize("K", [6, 10, 15])
def test_gemm_decomposition_reproduces_the_volume_contraction(lib, K):
    rng = np.random.default_rng(K)
    n = 7
    xi, U, V, u, v = (rng.standard_normal((n, K)) for _ in range(5))
    hb = rng.standard_normal((n, 3))
    J = rng.standard_normal((n, 4))
    rs = rng.uniform(0.5, 2.0, n)
    g = 9.81
    # the G values the images hold (sum of the parts), as a full symmetric tensor
    P, Sp, Pp = decode(K, swedg.tc_operand_image(K))
    BS = sum(a.astype(np.float64) for a in Sp)[:K, :2 * P]
    BP = sum(a.astype(np.float64) for a in Pp)[:, :P]
    Gm = np.zeros((2, K, K, K))
    for k in range(2):
        for pr, (i, j) in enumerate(pairs(K)):
            Gm[k, :, i, j] = Gm[k, :, j, i] = BS[:, k * P + pr]
            assert np.array_equal(BP[16 * k:16 * k + K, pr], BS[:, k * P + pr])
    mask = np.array([[[used(q, i, j) for j in range(K)] for i in range(K)] for q in range(K)])
    assert not np.any(Gm[:, ~mask])
    # direct contraction (non-base triples only), physical gradients through J^-1
    pp = 0.5 * xi
    pp[:, :3] += hb
    uc = J[:, [0]] * u + J[:, [1]] * v
    vc = J[:, [2]] * u + J[:, [3]] * v
    Px = np.einsum("qij,ei,ej->eq", Gm[0], xi, pp)
    Py = np.einsum("qij,ei,ej->eq", Gm[1], xi, pp)
    rU = rs[:, None] * (np.einsum("qij,ei,ej->eq", Gm[0], U, uc) + np.einsum("qij,ei,ej->eq", Gm[1], U, vc)
                        + g * (J[:, [0]] * Px + J[:, [2]] * Py))
    rV = rs[:, None] * (np.einsum("qij,ei,ej->eq", Gm[0], V, uc) + np.einsum("qij,ei,ej->eq", Gm[1], V, vc)
                        + g * (J[:, [1]] * Px + J[:, [3]] * Py))
    # the kernel's GEMMs: symmetrised products x the images

    def sym(a, b):
        return np.stack([a[:, i] * b[:, j] + (a[:, j] * b[:, i] if i != j else 0.0) for i, j in pairs(K)], axis=1)

    AU = np.concatenate([sym(U, uc), sym(U, vc)], axis=1)
    AV = np.concatenate([sym(V, uc), sym(V, vc)], axis=1)
    # h_b's mean mode stays out of the P GEMM and is added as hb0 sum_i xi_i G_k[q][i][0]
    pp_tc = pp.copy()
    pp_tc[:, 0] -= hb[:, 0]
    AP = sym(xi, pp_tc)
    DU, DV, DP = AU @ BS.T, AV @ BS.T, AP @ BP.T
    DP[:, :K] += hb[:, [0]] * np.einsum("qi,ei->eq", Gm[0, :, :, 0], xi)
    DP[:, 16:16 + K] += hb[:, [0]] * np.einsum("qi,ei->eq", Gm[1, :, :, 0], xi)
    gU = rs[:, None] * (DU + g * (J[:, [0]] * DP[:, :K] + J[:, [2]] * DP[:, 16:16 + K]))
    gV = rs[:, None] * (DV + g * (J[:, [1]] * DP[:, :K] + J[:, [3]] * DP[:, 16:16 + K]))
    tol = 1e-9 * max(np.abs(rU).max(), np.abs(rV).max())
    assert np.abs(gU - rU).max() <= tol
    assert np.abs(gV - rV).max() <= tol
    assert np.abs(rU[:, 3:]).max() > 0.1  # the test exercises nonzero higher rows
