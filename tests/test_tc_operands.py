"""Host-side checks of the tensor-core volume contraction (precision mode
SWE_PREC_MIXED_TF32), no GPU: the library's constant operand images decode,
by the layout the header documents, to the oracle's G tensors of Eq. (13),
split into two TF32 parts; and the two-stage decomposition the kernel uses
(GEMMs of per-element velocity and pressure rows against those images, then
sums over the coefficient rows) reproduces the direct volume contraction of
the momentum rows."""
import numpy as np
import pytest

import oracle as O
from paper_2311_11348_gb300 import build, swedg

DEG = [0, 1, 1, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4]


@pytest.fixture(scope="module")
def lib():
    build.build()
    return swedg.load()


def at(r, c):  # K-major, 128-byte swizzle: 16-byte unit c/4 of row r at unit (c/4) ^ (r%8)
    return (r // 8) * 256 + (r % 8) * 32 + (((c // 4) ^ (r % 8)) * 4) + c % 4


def decode(K, img):
    """the two parts of the image as B[part][k][q][i][j]: row 16 i + q, column
    k K + j of a [16 K][32] operand per part; every other entry zero"""
    nb = 16 * K
    assert len(img) == 2 * nb * 32
    B = np.zeros((2, 2, 16, K, K), np.float32)
    seen = np.zeros(len(img), bool)
    for part in range(2):
        base = part * nb * 32
        for i in range(K):
            for q in range(16):
                for k in range(2):
                    for j in range(K):
                        o = base + at(16 * i + q, k * K + j)
                        B[part, k, q, i, j] = img[o]
                        seen[o] = True
    assert not np.any(img[~seen])  # the padding (q >= K, columns >= 2 K) is zero
    return B


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
    B = decode(K, swedg.tc_operand_image(K))
    G = O.tensors()["G"]
    assert np.all(B.view(np.uint32) & 0x1FFF == 0)  # every part is a TF32 value: no bits below the 10-bit mantissa
    S = B.astype(np.float64).sum(0)
    floor = 1e-14 * np.abs(G).max()  # the library's tables agree with the oracle's to this
    for k in range(2):
        for q in range(16):
            for i in range(K):
                for j in range(K):
                    want = G[k, q, i, j] if (q < K and used(q, i, j)) else 0.0
                    tol = 2.0 ** -21 * abs(want) + floor  # the parts sum to G within 2^-22 |G|
                    assert abs(S[k, q, i, j] - want) <= tol, (k, q, i, j)
                    if want:  # part 0 is G rounded to 10 mantissa bits
                        assert abs(B[0, k, q, i, j] - want) <= 2.0 ** -11 * abs(want) + floor


@pytest.mark.parametrize("K", [6, 10, 15])
def test_gemm_decomposition_reproduces_the_volume_contraction(lib, K):
    """the kernel's two stages: GEMMs of per-element rows (2 K values: the
    contravariant velocities, or g J^-1 xi / 2) against the image, giving W,
    ZU, ZV [i][q]; then the sums over i with the element's U, V, xi, and the
    bottom term's products with the higher elevation modes added apart"""
    rng = np.random.default_rng(K)
    n = 7
    xi, U, V, u, v = (rng.standard_normal((n, K)) for _ in range(5))
    hb = rng.standard_normal((n, 3))
    J = rng.standard_normal((n, 4))
    rs = rng.uniform(0.5, 2.0, n)
    g = 9.81
    B = decode(K, swedg.tc_operand_image(K)).astype(np.float64).sum(0)  # [k][q][i][j], q < 16
    Gm = B[:, :K]
    mask = np.array([[[used(q, i, j) for j in range(K)] for i in range(K)] for q in range(K)])
    assert not np.any(Gm[:, ~mask])
    # direct contraction (non-base triples only), physical gradients through J^-1;
    # the bottom term xi_i h_b_j only with a higher elevation mode i >= 3
    pp = 0.5 * xi
    uc = J[:, [0]] * u + J[:, [1]] * v
    vc = J[:, [2]] * u + J[:, [3]] * v
    Px, Py = (np.array([sum(xi[e, i] * (pp[e, j] + (hb[e, j] if i >= 3 and j < 3 else 0.0)) * Gm[k][:, i, j]
                            for i in range(K) for j in range(K)) for e in range(n)]) for k in range(2))
    rU = rs[:, None] * (np.einsum("qij,ei,ej->eq", Gm[0], U, uc) + np.einsum("qij,ei,ej->eq", Gm[1], U, vc)
                        + g * (J[:, [0]] * Px + J[:, [2]] * Py))
    rV = rs[:, None] * (np.einsum("qij,ei,ej->eq", Gm[0], V, uc) + np.einsum("qij,ei,ej->eq", Gm[1], V, vc)
                        + g * (J[:, [1]] * Px + J[:, [3]] * Py))
    # the kernel: the operand B[(i, q)][(k, j)] and three A operands of 2 K columns
    Bop = np.zeros((16 * K, 2 * K))
    for i in range(K):
        for q in range(16):
            Bop[16 * i + q, :K] = B[0, q, i, :]
            Bop[16 * i + q, K:] = B[1, q, i, :]
    Aw = np.hstack([uc, vc])
    Au = g * np.hstack([J[:, [0]] * pp, J[:, [2]] * pp])
    Av = g * np.hstack([J[:, [1]] * pp, J[:, [3]] * pp])
    W, ZU, ZV = ((A @ Bop.T).reshape(n, K, 16) for A in (Aw, Au, Av))
    ex = np.einsum("qij,ei,ej->eq", Gm[0, :, 3:, :3], xi[:, 3:], hb)
    ey = np.einsum("qij,ei,ej->eq", Gm[1, :, 3:, :3], xi[:, 3:], hb)
    gU = np.einsum("ei,eiq->eq", U, W) + np.einsum("ei,eiq->eq", xi, ZU)
    gV = np.einsum("ei,eiq->eq", V, W) + np.einsum("ei,eiq->eq", xi, ZV)
    gU = rs[:, None] * (gU[:, :K] + g * (J[:, [0]] * ex + J[:, [2]] * ey))
    gV = rs[:, None] * (gV[:, :K] + g * (J[:, [1]] * ex + J[:, [3]] * ey))
    tol = 1e-9 * max(np.abs(rU).max(), np.abs(rV).max())
    assert np.abs(gU - rU).max() <= tol
    assert np.abs(gV - rV).max() <= tol
    assert np.abs(rU[:, 3:]).max() > 0.1  # the test exercises nonzero higher rows
