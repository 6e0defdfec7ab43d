"""Algorithmic operation counts of the libswedg kernel families (bench roofline).

The counts mirror the arithmetic of the kernels (same loops, the same
compile-time sparsity predicates of the reference tensors): an FMA counts as
2 floating-point operations, an add, multiply, division or square root as 1;
loads, conversions and selects count 0.  They are the "algorithmic flops per
unit" of the roofline that bench.py reports:

  family      unit                         arithmetic       count per unit
  usolve      element (p<=1 / p>=2)        FP64 / corr      USOLVE_P1 / usolve_flops(K, rc)
  edge_base   edge                         FP64             EDGE_BASE
  elem_base   element                      FP64             ELEM_BASE (first stage ELEM_BASE_EULER)
  edge_corr   edge with max(p_L,p_R) >= 2  corr type        edge_corr_flops(K_L, K_R, pmax)
  elem_corr   element p >= 2               corr type        elem_corr_flops(K, tc, rc)
  vol_tc      element p >= 2               TF32 tensor      vol_tc_flops(K)

"corr type" is FP64 in the FP64 mode and FP32 in both mixed modes.  In the
FP64 and mixed modes the velocity solve of a p >= 2 element also forms the
volume terms of the degree-1 test modes (rc), and elem_corr covers the test
modes of degree >= 2; in the tensor-core mode ("tf32") elem_corr covers every
test mode and leaves the momentum volume terms of p >= 3 to vol_tc, whose
count is the MMA work it issues: three GEMMs (velocities, and the pressure
products for each momentum equation) against the 16 K x 2 K operand of G,
each in three TF32 passes (head x head, head x tail, tail x head) over the
reduction padded to a multiple of 8.  The CFL bounds (DT per element, first
stage of a step) are part of the usolve family.
"""
from __future__ import annotations

import numpy as np

DEG = [0, 1, 1, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4]
KP = [1, 3, 6, 10, 15]
SM_COUNT = 152
SM_MAX_GHZ = 2.07
# FP64 pipe of a GB300: 2 DFMA = 4 flop per clock per SM (measured 1.19 TFLOP/s at 1.92 GHz)
FP64_PEAK_TFLOPS = SM_COUNT * 4 * SM_MAX_GHZ / 1e3
# FP32 pipe: 128 FMA = 256 flop per clock per SM
FP32_PEAK_TFLOPS = SM_COUNT * 256 * SM_MAX_GHZ / 1e3
# dense TF32 : BF16 tensor rate of the part (1.1 : 2.25 PFLOP/s nominal)
TF32_OVER_BF16 = 1.1 / 2.25

USOLVE_P1 = 76   # the 3 x 3 solve with the entries the orthonormal basis fixes left out
EDGE_BASE = 152
ELEM_BASE = 226  # a stage with the full SSP-RK combination
ELEM_BASE_EULER = 199  # the first stage (c + dt r)
DT = 12


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


def usolve_flops(K, rc=False):
    """truncated K x K assembly, LDL^T, two right-hand sides (and, with rc,
    the volume terms of test modes 1 and 2)"""
    f = 3
    for j in range(K):
        for i in range(j + 1):
            f += 2 * sum(1 for n in range(ktr(i, j)) if tnz(n, i, j))
    for j in range(K):
        f += 3 * j + 1 + (K - 1 - j) * (3 * j + 1)
    f += 2 * (K * (K - 1) + K + K * (K - 1) + K)
    if rc:
        f += setup_flops(K) + sum(volume_flops(K, q) for q in (1, 2))
    return f


def setup_flops(K, tc=False):
    """contravariant coefficients (J^-1 applied to u, v and to U, V of degree < p) and xi/2"""
    KL = KP[DEG[K - 1] - 1]
    return KL * 6 if tc else K * 6 + KL * 6


def volume_flops(K, q, tc=False):
    """the volume contraction of test mode q (non-base triples); with tc only the elevation row"""
    f = 0
    for i in range(K):
        if dnz(q, i) and not (q < 3 and i < 3):
            f += 4
        if tc:
            continue
        inner = sum(1 for j in range(K) if gnz(q, i, j) and not (q < 3 and i < 3 and j < 3))
        # the bottom term's h_b_j (j < 3) joins the products of the higher elevation modes
        hb = sum(1 for j in range(3) if gnz(q, i, j)) if i >= 3 else 0
        f += 8 * inner + hb + (8 if inner else 0)
    return f + (0 if tc else 10)


def elem_corr_flops(K, tc=False, rc=True):
    """volume contraction (non-base triples), source, the three edges'
    projected fluxes and the RK combination of the higher test modes; with rc
    also test modes 1 and 2; with tc the momentum rows' volume terms are vol_tc's"""
    f = setup_flops(K, tc)
    for q in range(1 if rc else 3, K):
        f += volume_flops(K, q, tc)
        if q >= 3:
            f += 4 + 3 * 3 + 3 * 5
    return f


def vol_tc_flops(K):
    """TF32 MMA flops per element (row of the GEMMs): three GEMMs of N = 16 K
    columns (rows i, test modes q padded to 16) over ceil(2K / 8) steps of 8,
    each in three passes (hh, ht, th); 2 flops per multiply-add"""
    return 3 * 3 * 2 * (16 * K) * 8 * ((2 * K + 7) // 8)


def edge_corr_flops(KL, KR, pm):
    """traces of both sides (5 fields), lambda, the FP64 elevation jump at the
    edge ends, the flux and the jump term at npts(pm) points and the flux's two
    moments, the projections onto the higher test modes of each side"""
    N = npts(pm)
    f = 12 + 30 + N * (2 * 10 * (KL + KR) + (KL + KR) + 99)
    for K in (KL, KR):
        if K >= 6:
            f += (K - 3) * (8 * N + 7)
    return f


def family_flops(orders, fam, nedge=None, mode="mixed"):
    """flops per SSP-RK3 step (3 stages) of one kernel family on an order map"""
    p = np.asarray(orders)
    ne = len(p)
    n = [int((p == q).sum()) for q in range(5)]
    nedge = nedge or int(round(1.5 * ne))
    st = 3
    if fam == "elem_base":
        return ((st - 1) * ELEM_BASE + ELEM_BASE_EULER) * ne
    if fam == "edge_base":
        return st * EDGE_BASE * nedge
    if fam == "dt":
        return 0
    if fam == "usolve":
        rc = mode != "tf32"
        return st * (n[1] * USOLVE_P1 + n[0] * 6 + sum(n[q] * usolve_flops(KP[q], rc) for q in (2, 3, 4))) + DT * ne
    if fam == "elem_corr":
        return st * sum(n[q] * elem_corr_flops(KP[q], tc=(mode == "tf32" and q >= 3), rc=(mode == "tf32"))
                        for q in (2, 3, 4))
    if fam == "vol_tc":  # orders 3 and 4 (order 2 stays on the CUDA cores)
        return st * sum(n[q] * vol_tc_flops(KP[q]) for q in (3, 4))
    if fam == "edge_corr":
        # i.i.d. orders: an edge's pmax is the larger of two independent draws
        frac = np.array(n, float) / max(ne, 1)
        cdf = np.cumsum(frac)
        tot = 0.0
        for pm in (2, 3, 4):
            pr = cdf[pm] ** 2 - cdf[pm - 1] ** 2
            tot += pr * nedge * edge_corr_flops(KP[pm], KP[max(1, pm - 1)], pm)
        return st * tot
    return None


def pipe_of(fam, mode):
    """which arithmetic pipe bounds a family: 'fp64', 'fp32' or 'tensor'"""
    if fam == "vol_tc":
        return "tensor"
    if fam in ("edge_corr", "elem_corr") and mode in ("mixed", "tf32"):
        return "fp32"
    return "fp64"
