"""Algorithmic operation and byte counts of the libswedg kernel families.

The counts mirror the arithmetic the kernels perform (same loops, same
compile-time sparsity predicates of the reference tensors); an FMA counts
as 2 floating-point operations, a division or square root as 1.  They are
the "algorithmic flops per unit" of the roofline in bench.py:

  family      unit                          what one unit computes
  usolve      element                       truncated uH = q system (Sect. 3)
  edge_base   edge                          P1 traces + LF flux at 2 points
  edge_corr   correction edge (pmax >= 2)   traces + flux at npts(pmax) points
  elem_corr   element p >= 2 (+ p <= 1 elements next to a correction edge)
  elem_base   element                       volume, source, projections, RK

Bytes per unit count every array element the kernel reads or writes once
(perfect reuse of neighbour data in L2 is assumed for edges).
"""
from __future__ import annotations

import numpy as np

DEG = [0, 1, 1, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4]
KP = [1, 3, 6, 10, 15]
# FP64 pipe of a GB300: 152 SMs x 4 flop/clk (2 DFMA) x 2.07 GHz (max SM clock)
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
# FP32 pipe: 152 SMs x 128 FMA/clk x 2 x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 256 * 2.07e9 / 1e12


def npts(pm):
    return 2 if pm <= 1 else (3 * pm + 2) // 2


def gnz(q, i, j):
    dq, di, dj = DEG[q], DEG[i], DEG[j]
    if dq == 0:
        return False
    if dq == 1:
        return i == j
    return di <= dj + dq - 1 and dj <= di + dq - 1


def dnz(q, i):
    return DEG[i] < DEG[q] and (DEG[q] != 1 or i == 0)


def tnz(n, i, j):
    a, b, c = DEG[n], DEG[i], DEG[j]
    return a <= b + c and b <= a + c and c <= a + b


def ktr(i, j):
    return KP[max(DEG[i], DEG[j])]


def usolve_flops(K):
    if K <= 3:
        return 92 if K == 3 else 6
    f = 4  # H + h_b, depth check
    for j in range(K):
        for i in range(j + 1):
            f += 2 * sum(1 for n in range(15) if n < ktr(i, j) and tnz(n, i, j))
    for j in range(K):
        f += 3 * j + 1
        for i in range(j + 1, K):
            f += 3 * j + 1
    f += 2 * (2 * (K * (K - 1) // 2) * 2 + 2 * K)  # two right-hand sides: L, D, L^T, scale by s
    return f


def elem_corr_flops(K, edge_pms):
    f = 8 * K
    for q in range(K):
        for i in range(K):
            if dnz(q, i) and not (q < 3 and i < 3):
                f += 9
            inner = sum(1 for j in range(K) if gnz(q, i, j) and not (q < 3 and i < 3 and j < 3))
            f += 8 * inner + (8 if inner else 0)
        f += 12 + (4 if q >= 3 else 0)
    for pm in edge_pms:
        N = npts(pm)
        f += N * (3 + 3 * 3 * 2 + (K - 3) * 7)
    f += 3 * (K - 3) * 5
    return f


def edge_corr_flops(KL, KR, pm, interior=True):
    N = npts(pm)
    f = N * 11 * KL + (N * 11 * KR if interior else N * 30)
    return f + N * 100


ELEM_BASE = 258   # per element (stage with a != 0); see the module docstring
EDGE_BASE = 234   # per interior edge
DT = 20           # per element, first stage of a CFL step


def family_flops(orders, fam, mode="fp64", edges=None):
    """FP64 (fp64 mode) or FP64+FP32 flops per step of one kernel family."""
    p = np.asarray(orders)
    ne = len(p)
    n = [int((p == q).sum()) for q in range(5)]
    stages = 3
    if fam == "elem_base":
        return {"flops_per_step": stages * ELEM_BASE * ne, "unit": "element"}
    if fam == "edge_base":
        nedge = int(1.5 * ne)
        return {"flops_per_step": stages * EDGE_BASE * nedge, "unit": "edge"}
    if fam == "usolve":
        f = n[1] * 92 + n[0] * 6 + sum(n[q] * usolve_flops(KP[q]) for q in (2, 3, 4))
        return {"flops_per_step": stages * f, "unit": "element"}
    if fam == "elem_corr":
        f = sum(n[q] * elem_corr_flops(KP[q], [q] * 3) for q in (2, 3, 4))
        return {"flops_per_step": stages * f, "unit": "element"}
    if fam == "edge_corr":
        f = sum(n[q] * 1.5 * edge_corr_flops(KP[q], KP[q], q) for q in (2, 3, 4))
        return {"flops_per_step": stages * f, "unit": "edge"}
    return None
