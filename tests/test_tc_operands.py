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
    """the two parts of the image as Gx, Gy [part][16][K][16] (from the U/V
    operand) and Gp [part][2][16][K][16] (from the pressure operand)"""
    C = (K + 1) // 2
    bpart = C * (2 * 16 * 32 + 32 * 32)
    assert len(img) == 2 * bpart

    def at(r, c):  # K-major, 128-byte swizzle: 16-byte unit c/4 of row r at unit (c/4) ^ (r%8)
        return (r // 8) * 256 + (r % 8) * 32 + (((c // 4) ^ (r % 8)) * 4) + c % 4

    Gx = np.zeros((2, 16, K, 16), np.float32)
    Gy = np.zeros((2, 16, K, 16), np.float32)
    Gp = np.zeros((2, 2, 16, K, 16), np.float32)
    for part in range(2):
        base = part * bpart
        for i in range(K):
            c, col0 = i // 2, 16 * (i % 2)
            for q in range(16):
                for j in range(16):
                    Gx[part, q, i, j] = img[base + c * 512 + at(q, col0 + j)]
                    Gy[part, q, i, j] = img[base + (C + c) * 512 + at(q, col0 + j)]
                    for k in range(2):
                        Gp[part, k, q, i, j] = img[base + 2 * C * 512 + c * 1024 + at(16 * k + q, col0 + j)]
        if K % 2:  # the padding row of the last chunk is zero
            c = K // 2
            for q in range(16):
                for j in range(16):
                    assert img[base + c * 512 + at(q, 16 + j)] == 0
    return Gx, Gy, Gp


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
    Gx, Gy, Gp = decode(K, swedg.tc_operand_image(K))
    G = O.tensors()["G"]
    for a in (Gx, Gy, Gp):  # every part is a TF32 value: no bits below the 10-bit mantissa
        assert np.all(a.view(np.uint32) & 0x1FFF == 0)
    S = [Gx.astype(np.float64).sum(0), Gy.astype(np.float64).sum(0)]
    Pm = Gp.astype(np.float64).sum(0)
    floor = 1e-14 * np.abs(G).max()  # the library's tables agree with the oracle's to this
    for k in range(2):
        assert np.array_equal(Pm[k], S[k])  # both operands hold the same values
        for q in range(16):
            for i in range(K):
                for j in range(16):
                    want = G[k, q, i, j] if (q < K and j < K and used(q, i, j)) else 0.0
                    tol = 2.0 ** -21 * abs(want) + floor  # the parts sum to G within 2^-22 |G|
                    assert abs(S[k][q, i, j] - want) <= tol, (k, q, i, j)
                    if want:  # part 0 is G rounded to 10 mantissa bits
                        part0 = (Gx if k == 0 else Gy)[0, q, i, j]
                        assert abs(part0 - want) <= 2.0 ** -11 * abs(want) + floor


@pytest.mark.parametrize("K", [6, 10, 15])
def test_gemm_decomposition_reproduces_the_volume_contraction(lib, K):
    rng = np.random.default_rng(K)
    n = 7
    xi, U, V, u, v = (rng.standard_normal((n, K)) for _ in range(5))
    hb = rng.standard_normal((n, 3))
    J = rng.standard_normal((n, 4))
    rs = rng.uniform(0.5, 2.0, n)
    g = 9.81
    # the G values the images hold (sum of the parts)
    Gx, Gy, Gp = decode(K, swedg.tc_operand_image(K))
    Gm = np.stack([Gx.astype(np.float64).sum(0)[:K, :, :K], Gy.astype(np.float64).sum(0)[:K, :, :K]])
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
    # the kernel's GEMMs: rows i x 16 columns j of coefficient products against the images
    def rows(a, b):
        bb = np.zeros((n, 16))
        bb[:, :K] = b
        return (a[:, :, None] * bb[:, None, :]).reshape(n, K * 16)

    BSx = Gx.astype(np.float64).sum(0)[:K].reshape(K, K * 16)
    BSy = Gy.astype(np.float64).sum(0)[:K].reshape(K, K * 16)
    BPx = Gp[:, 0].astype(np.float64).sum(0)[:K].reshape(K, K * 16)
    BPy = Gp[:, 1].astype(np.float64).sum(0)[:K].reshape(K, K * 16)
    DU = rows(U, uc) @ BSx.T + rows(U, vc) @ BSy.T
    DV = rows(V, uc) @ BSx.T + rows(V, vc) @ BSy.T
    # h_b's mean mode stays out of the pressure GEMM and is added as hb0 sum_i xi_i G_k[q][i][0]
    pp_tc = pp.copy()
    pp_tc[:, 0] -= hb[:, 0]
    DPx = rows(xi, pp_tc) @ BPx.T + hb[:, [0]] * np.einsum("qi,ei->eq", Gm[0, :, :, 0], xi)
    DPy = rows(xi, pp_tc) @ BPy.T + hb[:, [0]] * np.einsum("qi,ei->eq", Gm[1, :, :, 0], xi)
    DP = np.zeros((n, 32))
    DP[:, :K], DP[:, 16:16 + K] = DPx, DPy
    gU = rs[:, None] * (DU + g * (J[:, [0]] * DP[:, :K] + J[:, [2]] * DP[:, 16:16 + K]))
    gV = rs[:, None] * (DV + g * (J[:, [1]] * DP[:, :K] + J[:, [3]] * DP[:, 16:16 + K]))
    tol = 1e-9 * max(np.abs(rU).max(), np.abs(rV).max())
    assert np.abs(gU - rU).max() <= tol
    assert np.abs(gV - rV).max() <= tol
    assert np.abs(rU[:, 3:]).max() > 0.1  # the test exercises nonzero higher rows
