"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the DG method: it makes triangulations,
vertex bathymetry, initial-condition functions and per-element order maps.
It serves the CUDA path, the oracle, the tests and the benchmark alike.

Workloads (the paper measures a dam break on a randomly perturbed uniform
mesh of 2,097,152 triangles and a tidal flow with a block-structured mesh,
Sect. 5; neither mesh nor bathymetry is available, so these are synthetic
stand-ins with the paper's mesh sizes and order fractions):

  unit_p1     [0,1]^2, 16x16 split squares (512 triangles), p = 1,
              h_b = 1 + 0.1 sin(2 pi x) cos(2 pi y),
              xi0 = 0.01 exp(-((x-.5)^2 + (y-.5)^2)/0.01), land walls.
  ocean_p123  [0,1e5]^2 m, 256x256 split squares (131,072 triangles) with
              +-20% interior vertex jitter (seed 2), Fourier bathymetry
              50..4000 m (32 modes, seed 3), Gaussian hump of 1 m and
              sigma = 5 km, orders p in {1,2,3} (70/20/10 %, seed 5), walls.
  shelf_p1234 [0,5e5]^2 m, 1024x1024 split squares (2,097,152 triangles),
              tanh shelf 4000 m -> 20 m with 2 % Fourier noise (seed 4),
              elliptic 3 m elevation, M2 tide (1 m, 44714 s) on x = 0,
              orders p in {1..4} (40/30/20/10 %, seed 5).
"""
from __future__ import annotations

import math

import numpy as np


def split_square_mesh(n: int, L: float = 1.0, x0: float = 0.0, y0: float = 0.0, jitter: float = 0.0,
                      seed: int = 0):
    """n x n squares of side L/n, each cut along its (i,j)->(i+1,j+1) diagonal.

    Returns (xy[nv,2] float64, tri[ne,3] int32), triangles counter-clockwise,
    2 n^2 triangles.  Interior vertices move by U[-jitter h, jitter h]^2."""
    h = L / n
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    xy = np.stack([x0 + i.ravel() * h, y0 + j.ravel() * h], axis=1).astype(np.float64)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter * h, jitter * h, size=xy.shape)
        inner = ((i.ravel() > 0) & (i.ravel() < n) & (j.ravel() > 0) & (j.ravel() < n))
        xy[inner] += d[inner]
    vid = lambda a, b: a * (n + 1) + b  # noqa: E731
    a, b = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    a = a.ravel(); b = b.ravel()
    v00, v10, v11, v01 = vid(a, b), vid(a + 1, b), vid(a + 1, b + 1), vid(a, b + 1)
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    tri = np.empty((2 * n * n, 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2
    return xy, tri


def boundary_tags(xy, tri, open_side=None, tol=1e-9):
    """[ne,3] tags for the edge opposite each vertex: 0 interior/land,
    2 open sea on the side x = min x when open_side == 'west'."""
    tags = np.zeros(tri.shape, dtype=np.int8)
    if open_side is None:
        return tags
    xmin = xy[:, 0].min()
    for k in range(3):
        a = tri[:, (k + 1) % 3]
        b = tri[:, (k + 2) % 3]
        if open_side == "west":
            on = (np.abs(xy[a, 0] - xmin) < tol) & (np.abs(xy[b, 0] - xmin) < tol)
        else:
            raise ValueError(open_side)
        tags[on, k] = 2
    return tags


def fourier_field(x, y, L, nmodes=32, kmax=8, seed=3):
    """S(x, y) = sum_m a_m cos(2 pi (k_m . x)/L + phi_m), k_m in {-kmax..kmax}^2 \\ 0,
    a_m ~ |k_m|^-1.5, phi_m ~ U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=2)
        if k[0] == 0 and k[1] == 0:
            continue
        ks.append(k)
    ks = np.array(ks, dtype=np.float64)
    amp = np.linalg.norm(ks, axis=1) ** -1.5
    ph = rng.uniform(0.0, 2.0 * math.pi, size=nmodes)
    S = np.zeros_like(x, dtype=np.float64)
    for m in range(nmodes):
        S += amp[m] * np.cos(2.0 * math.pi * (ks[m, 0] * x + ks[m, 1] * y) / L + ph[m])
    return S


def fourier_bathymetry(xy, L, lo=50.0, hi=4000.0, seed=3):
    S = fourier_field(xy[:, 0], xy[:, 1], L, seed=seed)
    return lo + (hi - lo) * (S - S.min()) / (S.max() - S.min())


def shelf_bathymetry(xy, L=5e5, seed=4):
    x = xy[:, 0]
    base = 20.0 + 3980.0 * 0.5 * (1.0 - np.tanh((x - 0.5 * L) / 2e4))
    S = fourier_field(xy[:, 0], xy[:, 1], L, seed=seed)
    noise = 2.0 * (S - S.min()) / (S.max() - S.min()) - 1.0
    return base * (1.0 + 0.02 * noise)


def orders_fractions(ne: int, fractions: dict, seed: int = 5):
    """i.i.d. seeded order map with the given fraction per order, e.g. {1: .7, 2: .2, 3: .1}."""
    rng = np.random.default_rng(seed)
    ps = np.array(sorted(fractions))
    pr = np.array([fractions[p] for p in ps], dtype=np.float64)
    return ps[rng.choice(len(ps), size=ne, p=pr / pr.sum())].astype(np.int8)


def orders_every_nth(ne: int, nth: int, p_lo: int, p_hi: int, offset: int = 0):
    """Static adaptivity of the paper's dam break: every nth element at p_hi."""
    p = np.full(ne, p_lo, dtype=np.int8)
    p[offset::nth] = p_hi
    return p


# ---------------- the three single-mesh workloads ----------------

def unit_p1():
    xy, tri = split_square_mesh(16, 1.0)
    hv = 1.0 + 0.1 * np.sin(2 * math.pi * xy[:, 0]) * np.cos(2 * math.pi * xy[:, 1])

    def ic(x, y):
        return 0.01 * np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2) / 0.01), 0.0 * x, 0.0 * x

    return dict(name="unit_p1", xy=xy, tri=tri, hv=hv, orders=np.ones(len(tri), np.int8), ic=ic,
                bc_tag=None, g=9.81, rk_order=2, cfl=0.1, steps=200)


def ocean_p123(n: int = 256, fractions=None):
    L = 1e5
    xy, tri = split_square_mesh(n, L, jitter=0.2, seed=2)
    hv = fourier_bathymetry(xy, L, seed=3)
    fr = fractions or {1: 0.7, 2: 0.2, 3: 0.1}

    def ic(x, y):
        r2 = (x - 0.5 * L) ** 2 + (y - 0.5 * L) ** 2
        return np.exp(-r2 / (2.0 * 5000.0 ** 2)), 0.0 * x, 0.0 * x

    return dict(name=f"ocean_p123_n{n}", xy=xy, tri=tri, hv=hv, orders=orders_fractions(len(tri), fr, seed=5),
                ic=ic, bc_tag=None, g=9.81, rk_order=3, cfl=0.1, steps=1000)


def shelf_p1234(n: int = 1024):
    L = 5e5
    xy, tri = split_square_mesh(n, L)
    hv = shelf_bathymetry(xy, L, seed=4)

    def ic(x, y):
        return 3.0 * np.exp(-((x - 3e5) / 4e4) ** 2 - ((y - 2.5e5) / 1.5e4) ** 2), 0.0 * x, 0.0 * x

    return dict(name=f"shelf_p1234_n{n}", xy=xy, tri=tri, hv=hv,
                orders=orders_fractions(len(tri), {1: 0.4, 2: 0.3, 3: 0.2, 4: 0.1}, seed=5),
                ic=ic, bc_tag=boundary_tags(xy, tri, "west"), g=9.81, rk_order=3, cfl=0.1, steps=5000,
                tide=(1.0, 44714.0, 0.0))


def dam_break_p12(n: int = 1024, nth: int = 32, L: float = 1e4, seed: int = 9):
    """The paper's radial dam break setting (Sect. 5): a randomly perturbed
    uniform mesh of 2 n^2 triangles (2,097,152 at n = 1024) over a flat bottom
    (10 m), a circular dam of radius L/8 holding 1 m of extra water (a smooth
    tanh step 20 m wide), walls; static adaptivity p1-2 with every nth element
    at p = 2 (nth = 0: p = 1 everywhere, nth = 1: p = 2 everywhere)."""
    xy, tri = split_square_mesh(n, L, jitter=0.2, seed=seed)
    hv = np.full(len(xy), 10.0)
    ne = len(tri)
    if nth == 0:
        orders = np.full(ne, 1, dtype=np.int8)
    else:
        orders = orders_every_nth(ne, nth, 1, 2)

    def ic(x, y):
        r = np.sqrt((x - 0.5 * L) ** 2 + (y - 0.5 * L) ** 2)
        return 0.5 * (1.0 - np.tanh((r - L / 8) / 20.0)), 0.0 * x, 0.0 * x

    return dict(name=f"dam_break_p12_n{n}_nth{nth}", xy=xy, tri=tri, hv=hv, orders=orders, ic=ic,
                bc_tag=None, g=9.81, rk_order=3, cfl=0.1)


# ---------------- many-mesh workloads ----------------

def _member(T: float, seed: int, L: float = 1e5, fractions=None):
    """one ocean-like member of about T triangles: its own jitter, Fourier
    bathymetry (50..4000 m), order map and Gaussian hump (1 m, sigma = 5 % of L)"""
    n = max(2, int(round(math.sqrt(T / 2.0))))
    xy, tri = split_square_mesh(n, L, jitter=0.2, seed=seed)
    hv = fourier_bathymetry(xy, L, seed=seed + 1)
    orders = orders_fractions(len(tri), fractions or {1: 0.4, 2: 0.3, 3: 0.2, 4: 0.1}, seed=seed + 2)
    cx, cy = np.random.default_rng(seed + 3).uniform(0.3 * L, 0.7 * L, size=2)
    sig = 0.05 * L
    xi_v = np.exp(-((xy[:, 0] - cx) ** 2 + (xy[:, 1] - cy) ** 2) / (2.0 * sig * sig))
    return dict(xy=xy, tri=tri, hv=hv, orders=orders, xi_vertex=xi_v)


def log_uniform_sizes(count: int, lo: float, hi: float, seed: int):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))


def ensemble_members(count: int = 64, lo: float = 8e3, hi: float = 6e5, seed: int = 6):
    """Batched ensemble: `count` members with triangle counts log-uniform in
    [lo, hi] (seeded), each an ocean-like member with orders p in {1..4}
    (40/30/20/10 %).  Each dict has xy, tri, hv, orders and xi_vertex (the
    initial elevation at the vertices; momenta start at rest)."""
    sizes = log_uniform_sizes(count, lo, hi, seed)
    return [_member(T, 1000 * seed + 10 * m) for m, T in enumerate(sizes)]


def serving_requests(rate: float, duration: float, lo: float = 5e3, hi: float = 2e6, steps_lo: int = 100,
                     steps_hi: int = 2000, seed: int = 7, pool: int = 0):
    """Poisson arrivals at `rate` per second over `duration` seconds; each
    request an ensemble-style member of log-uniform [lo, hi] triangles with a
    step count uniform in [steps_lo, steps_hi].  Returns a list of
    (arrival offset in s, member dict, steps).  pool > 0: the members are
    drawn (uniformly, seeded) from `pool` members generated once with
    log-uniform sizes, so that thousands of requests need no thousands of
    mesh generations; the requests still run as independent simulations."""
    rng = np.random.default_rng(seed)
    members = []
    if pool > 0:
        prng = np.random.default_rng(seed + 1)
        sizes = np.exp(prng.uniform(math.log(lo), math.log(hi), size=pool))
        members = [_member(T, 7000 + 10 * k) for k, T in enumerate(sizes)]
    out = []
    t = rng.exponential(1.0 / rate)
    k = 0
    while t < duration:
        T = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        m = members[int(rng.integers(pool))] if pool > 0 else _member(T, 7000 + 10 * k)
        out.append((t, m, steps))
        t += rng.exponential(1.0 / rate)
        k += 1
    return out
