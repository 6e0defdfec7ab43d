"""Pins of the oracle's scheme (no GPU): the right-hand side of Eq. (8) with
the Lax-Friedrichs flux and Eq. (10), the truncated auxiliary system of
Sect. 3, the order separation of Sect. 3 and the SSP-RK time stepping.

Every check compares the oracle with something other than itself:
brute-force quadrature of the pointwise weak form, a separate finite-volume
code, exact invariants (mass, lake at rest, free stream, rotation) and the
order of accuracy in time.
"""
import math

import numpy as np
import pytest

import dgref
import oracle as O
from paper_2311_11348_gb300 import inputs

K_OF_P = dgref.K_OF_P


def tiny_meshes():
    one = (np.array([[0.1, 0.0], [1.3, 0.2], [0.4, 0.9]]), np.array([[0, 1, 2]]))
    two = (np.array([[0.0, 0.0], [1.0, 0.1], [1.1, 1.0], [-0.1, 0.9]]), np.array([[0, 1, 2], [0, 2, 3]]))
    xy, tri = inputs.split_square_mesh(2, 1.0, jitter=0.2, seed=11)
    tri = tri.copy()
    tri[3] = tri[3][[0, 2, 1]]  # one clockwise triangle: must be re-oriented
    return [one, two, (xy, tri)]


def random_state(ne, orders, rng, mean_xi=0.3, amp=0.05):
    c = np.zeros((3, 15, ne))
    for e in range(ne):
        K = K_OF_P[orders[e]]
        c[0, 0, e] = mean_xi
        c[0, 1:K, e] = amp * rng.standard_normal(K - 1) * 0.5 ** dgref.DEG[1:K]
        c[1, :K, e] = amp * rng.standard_normal(K) * 0.5 ** dgref.DEG[:K]
        c[2, :K, e] = amp * rng.standard_normal(K) * 0.5 ** dgref.DEG[:K]
    return c


def scale_state_means(c, area):
    c = c.copy()
    c[:, 0, :] *= np.sqrt(area)  # coefficient of a constant = value * sqrt|Omega|
    return c


def rhs_pin_errors(Om, case, seed):
    """(u error, rhs error), each relative to max(1, the reference's largest
    entry), of the oracle `Om` against the independent quadrature assembly of
    the truncated auxiliary system and the brute-force pointwise weak form, on
    tiny mesh `case` with orders 0..4 (case 1, seed 1: one open-sea edge)"""
    xy, tri = tiny_meshes()[case]
    rng = np.random.default_rng(100 * case + seed)
    ne = len(tri)
    orders = rng.integers(0, 5, size=ne).astype(np.int8)
    hv = 1.0 + 0.3 * rng.uniform(size=len(xy))
    bc = None
    opened = []
    if case == 1 and seed == 1:
        # the edge opposite vertex 1 of triangle 0 is (2,0): interior; make a boundary one open
        bc = np.zeros((ne, 3), np.int8)
        bc[0, 2] = 2  # edge opposite vertex 2: (0,1), on the boundary
        opened = [(0, 2)]
    g = 9.81
    m = Om.Mesh(xy, tri, hv, orders, bc_tag=bc)
    geo = m.geometry()
    c = scale_state_means(random_state(ne, orders, rng), geo["area"])
    P = Om.Params(g=g, tide_amp=0.05, tide_period=0.0)
    r, u = m.rhs(P, c, t=0.0, with_u=True)
    msh = dgref.Tri(xy, tri)
    u_ref = dgref.solve_u(msh, hv, orders, c)
    # the brute-force side orients triangles itself; element order is the same
    rb = dgref.brute_force_rhs(msh, hv, orders, c, u, g, bc_open=opened, xi_hat=0.05)
    return (np.abs(u - u_ref).max() / max(1.0, np.abs(u_ref).max()),
            np.abs(r - rb).max() / max(1.0, np.abs(rb).max()))


@pytest.mark.parametrize("case", range(3))
@pytest.mark.parametrize("seed", [0, 1])
def test_rhs_equals_brute_force_weak_form(case, seed):
    eu, er = rhs_pin_errors(O, case, seed)
    assert eu <= 1e-13 and er <= 1e-12, (eu, er)


def source_pin_errors(Om, case):
    """(rhs error relative to max(1, the reference's largest entry), size of the
    source's share of the rhs) of the oracle `Om` with bottom friction and
    Coriolis against the brute-force pointwise weak form on tiny mesh `case`"""
    xy, tri = tiny_meshes()[case]
    rng = np.random.default_rng(40 + case)
    ne = len(tri)
    orders = rng.integers(0, 5, size=ne).astype(np.int8)
    hv = 1.0 + 0.3 * rng.uniform(size=len(xy))
    g = 9.81
    m = Om.Mesh(xy, tri, hv, orders)
    geo = m.geometry()
    c = scale_state_means(random_state(ne, orders, rng), geo["area"])
    c[1, 0] += 0.4 * np.sqrt(geo["area"])  # a mean flow, so that |u| matters
    fr = dict(fric_lin=0.7, fric_quad=2.0, f_c=0.9)
    r, u = m.rhs(Om.Params(g=g, **fr), c, t=0.0, with_u=True)
    r0 = m.rhs(Om.Params(g=g), c, t=0.0)
    msh = dgref.Tri(xy, tri)
    rb = dgref.brute_force_rhs(msh, hv, orders, c, u, g, **fr)
    return np.abs(r - rb).max() / max(1.0, np.abs(rb).max()), np.abs(r - r0).max()


@pytest.mark.parametrize("case", range(3))
def test_friction_and_coriolis_equal_brute_force_weak_form(case):
    """Source of Eq. (5) with bottom friction from the element means (Sect. 3):
    the oracle against quadrature of the pointwise source on tiny meshes,
    orders 0..4 (coefficients inflated so that the source terms dominate)."""
    err, size = source_pin_errors(O, case)
    assert size > 1e-2  # the source terms are exercised
    assert err <= 1e-12, err


def test_friction_and_coriolis_closed_form_on_a_free_stream():
    """Uniform flow over a flat bottom: every flux cancels, and the rhs of the
    mean mode is the pointwise source (-tau u + f_c V, -tau v - f_c U) times
    sqrt|Omega| with tau = fric_lin H + fric_quad |u| (Eq. 5)."""
    xy, tri, hv, orders = jittered_mixed(seed=9)
    H0, xi0, U0, V0 = 3.0, 0.2, 0.5, -0.3
    hv = np.full(len(xy), H0 - xi0)
    m = O.Mesh(xy, tri, hv, orders)
    sa = np.sqrt(m.geometry()["area"])
    ne = len(tri)
    c = np.zeros((3, 15, ne))
    c[0, 0], c[1, 0], c[2, 0] = xi0 * sa, U0 * sa, V0 * sa
    fl, fq, fc = 1e-4, 0.009, 3.19e-5
    r = m.rhs(O.Params(g=9.81, fric_lin=fl, fric_quad=fq, f_c=fc), c)
    u0, v0 = U0 / H0, V0 / H0
    tau = fl * H0 + fq * np.hypot(u0, v0)
    inner = np.all(m.neighbours()["bc"] == 0, axis=1)
    # the fluxes cancel to round-off (1e-12 as in the free-stream pin), the source is ~4e-5
    assert np.allclose(r[1, 0, inner], (-tau * u0 + fc * V0) * sa[inner], rtol=0, atol=1e-12)
    assert np.allclose(r[2, 0, inner], (-tau * v0 - fc * U0) * sa[inner], rtol=0, atol=1e-12)
    assert np.abs((-tau * u0 + fc * V0) * sa).min() > 1e-5
    assert np.abs(r[0, :, inner]).max() < 1e-12 and np.abs(r[:, 1:, inner]).max() < 1e-12


def fv_rhs(xy, tri, hv, means, g):
    """First-order finite volumes with the paper's LF flux (lambda of Eq. 10
    from cell means), pressure g xi (xi/2 + h_b(x_E)) |E| and source
    g xi grad h_b |Omega| -- the p = 0 case of the scheme written out."""
    ne = len(tri)
    xi, U, V = means
    area = np.zeros(ne); grad = np.zeros((ne, 2)); hmean = np.zeros(ne)
    edges = {}
    for e in range(ne):
        a, b, c = xy[tri[e]]
        area[e] = 0.5 * abs((b[0] - a[0]) * (c[1] - a[1]) - (c[0] - a[0]) * (b[1] - a[1]))
        A = np.array([[b[0] - a[0], b[1] - a[1]], [c[0] - a[0], c[1] - a[1]]])
        h = hv[tri[e]]
        grad[e] = np.linalg.solve(A, [h[1] - h[0], h[2] - h[0]])
        hmean[e] = h.mean()
        for k in range(3):
            i, j = tri[e, (k + 1) % 3], tri[e, (k + 2) % 3]
            edges.setdefault((min(i, j), max(i, j)), []).append(e)
    H = xi + hmean
    uu, vv = U / H, V / H
    d = np.zeros((3, ne))
    cen = np.array([xy[t].mean(axis=0) for t in tri])
    for (i, j), els in edges.items():
        pa, pb = xy[i], xy[j]
        L = np.hypot(*(pb - pa))
        hm = 0.5 * (hv[i] + hv[j])
        e = els[0]
        n = np.array([pb[1] - pa[1], -(pb[0] - pa[0])]) / L
        if n @ (0.5 * (pa + pb) - cen[e]) < 0:
            n = -n
        ca = np.array([xi[e], U[e], V[e]])
        wa = np.array([uu[e], vv[e]])
        if len(els) == 2:
            f = els[1]
            cb = np.array([xi[f], U[f], V[f]]); wb = np.array([uu[f], vv[f]])
        else:
            qn = ca[1] * n[0] + ca[2] * n[1]
            cb = np.array([ca[0], ca[1] - 2 * qn * n[0], ca[2] - 2 * qn * n[1]])
            wb = wa - 2 * (wa @ n) * n
        lam = max(abs(wa @ n), abs(wb @ n)) + max(math.sqrt(g * (ca[0] + hm)), math.sqrt(g * (cb[0] + hm)))

        def flux(c_, w_):
            P = g * c_[0] * (0.5 * c_[0] + hm)
            un = w_ @ n
            return np.array([c_[1] * n[0] + c_[2] * n[1], c_[1] * un + P * n[0], c_[2] * un + P * n[1]])

        F = 0.5 * (flux(ca, wa) + flux(cb, wb) + lam * (ca - cb)) * L
        d[:, e] -= F
        if len(els) == 2:
            d[:, els[1]] += F
    d[1] += g * xi * grad[:, 0] * area
    d[2] += g * xi * grad[:, 1] * area
    return d / area


def test_mesh_geometry_closed_forms():
    """per element: |Omega_e| = the shoelace area, s_e = sqrt(2 |Omega_e|)
    (sqrt |det J_e|), the gradient of a linear bathymetry a + b x + c y is
    (b, c) exactly, and its three P1 modes are those of that plane: the
    element mean times sqrt|Omega_e| in mode 0"""
    rng = np.random.default_rng(31)
    xy, tri = inputs.split_square_mesh(5, 3.0, jitter=0.25, seed=31)
    tri = tri.astype(np.int32)
    flip = rng.uniform(size=len(tri)) < 0.5
    tri[flip] = tri[flip][:, [0, 2, 1]]
    a0, b0, c0 = 40.0, -3.0, 5.5
    hv = a0 + b0 * xy[:, 0] + c0 * xy[:, 1]
    m = O.Mesh(xy, tri, hv, np.ones(len(tri), np.int8))
    geo = m.geometry()
    P = xy[tri]
    area = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1])
                        - (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))
    assert np.allclose(geo["area"], area, rtol=1e-14, atol=0)
    assert np.allclose(geo["s"], np.sqrt(2.0 * area), rtol=1e-14, atol=0)
    assert np.allclose(geo["dhb"], np.tile([b0, c0], (len(tri), 1)), rtol=0, atol=1e-12)
    centroid = P.mean(axis=1)
    mean = a0 + b0 * centroid[:, 0] + c0 * centroid[:, 1]
    assert np.allclose(geo["hb"][:, 0], mean * np.sqrt(area), rtol=1e-13, atol=0)


def test_neighbour_map_equals_brute_force_pairing():
    """the oracle's mesh set-up: clockwise triangles re-oriented (a permutation
    of the given vertices with positive area), the neighbour map and local
    edge indices of the re-oriented triangles equal a brute-force pairing of
    their edges, boundary edges land unless tagged open sea"""
    rng = np.random.default_rng(21)
    xy, tri = inputs.split_square_mesh(6, 1.0, jitter=0.2, seed=21)
    tri = tri[rng.permutation(len(tri))].astype(np.int32)
    flip = rng.uniform(size=len(tri)) < 0.4
    tri[flip] = tri[flip][:, [0, 2, 1]]
    bc = inputs.boundary_tags(xy, tri, "west")
    m = O.Mesh(xy, tri, np.ones(len(xy)), np.ones(len(tri), np.int8), bc_tag=bc)
    nb = m.neighbours()
    t = nb["tri"]
    assert np.array_equal(np.sort(t, axis=1), np.sort(tri, axis=1))
    a, b, c = xy[t[:, 0]], xy[t[:, 1]], xy[t[:, 2]]
    assert np.all((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]) > 0)
    rb, rk = dgref.brute_force_adjacency(t)
    assert np.array_equal(nb["nb"], rb) and np.array_equal(nb["nbk"], rk)
    boundary = rb < 0
    assert np.all(nb["bc"][~boundary] == 0)
    # tags follow the caller's local edge numbering: edge k opposite vertex k of the given triangle
    open_edges = set()
    for e, k in zip(*np.nonzero(bc == 2)):
        open_edges.add((e, frozenset((int(tri[e][(k + 1) % 3]), int(tri[e][(k + 2) % 3])))))
    assert len(open_edges) == 6
    for e, k in zip(*np.nonzero(boundary)):
        key = (e, frozenset((int(t[e][(k + 1) % 3]), int(t[e][(k + 2) % 3]))))
        assert nb["bc"][e, k] == (2 if key in open_edges else 1)


def test_p0_is_first_order_finite_volumes():
    xy, tri = inputs.split_square_mesh(6, 2.0, jitter=0.2, seed=3)
    ne = len(tri)
    rng = np.random.default_rng(7)
    hv = 2.0 + 0.5 * rng.uniform(size=len(xy))
    m = O.Mesh(xy, tri, hv, np.zeros(ne, np.int8))
    area = m.geometry()["area"]
    means = np.stack([0.2 * rng.standard_normal(ne), 0.3 * rng.standard_normal(ne), 0.3 * rng.standard_normal(ne)])
    c = np.zeros((3, 15, ne))
    c[:, 0, :] = means * np.sqrt(area)
    r = m.rhs(O.Params(g=9.81), c)
    dg = r[:, 0, :] / np.sqrt(area)
    fv = fv_rhs(xy, tri, hv, means, 9.81)
    assert np.abs(dg - fv).max() <= 1e-13 * np.abs(fv).max()
    assert np.all(r[:, 1:, :] == 0.0)


def jittered_mixed(n=6, seed=4, pmin=0, pmax=4):
    xy, tri = inputs.split_square_mesh(n, 1.0, jitter=0.2, seed=seed)
    rng = np.random.default_rng(seed)
    orders = rng.integers(pmin, pmax + 1, size=len(tri)).astype(np.int8)
    hv = 1.0 + 0.2 * np.sin(3 * xy[:, 0]) * np.cos(2 * xy[:, 1])
    return xy, tri, hv, orders


@pytest.mark.parametrize("xi0", [0.0, 0.37])
def test_lake_at_rest(xi0):
    xy, tri, hv, orders = jittered_mixed()
    m = O.Mesh(xy, tri, hv, orders)
    area = m.geometry()["area"]
    c = np.zeros((3, 15, len(tri)))
    c[0, 0, :] = xi0 * np.sqrt(area)
    P = O.Params(g=9.81, rk_order=3, cfl=0.2)
    r = m.rhs(P, c)
    scale = 9.81 * max(xi0, 1.0) * hv.max()
    if xi0 == 0.0:
        assert np.all(r == 0.0)
    else:
        assert np.abs(r).max() <= 1e-12 * scale
    c1, t = m.run(P, c, 0.0, 1000)
    assert np.abs(c1 - c).max() <= 1e-12 * max(xi0, 1.0)


def test_free_stream_flat_bottom():
    xy, tri, hv, orders = jittered_mixed(seed=5)
    hv = np.full(len(xy), 3.0)
    m = O.Mesh(xy, tri, hv, orders)
    area = m.geometry()["area"]
    ne = len(tri)
    c = np.zeros((3, 15, ne))
    c[0, 0] = 0.2 * np.sqrt(area); c[1, 0] = 0.5 * np.sqrt(area); c[2, 0] = -0.3 * np.sqrt(area)
    r, u = m.rhs(O.Params(g=9.81), c, with_u=True)
    # constant H: u = U / H exactly (P10)
    assert np.allclose(u[0, 0] / np.sqrt(area), 0.5 / 3.2, rtol=1e-14, atol=0)
    assert np.abs(u[:, 1:]).max() < 1e-15
    nb = m.neighbours()["bc"]
    inner = np.all(nb == 0, axis=1)
    assert inner.sum() > 10
    assert np.abs(r[:, :, inner]).max() < 1e-12


def test_usolve_constant_depth_any_momentum():
    xy, tri, hv, orders = jittered_mixed(seed=6, pmin=1)
    hv = np.full(len(xy), 2.5)
    m = O.Mesh(xy, tri, hv, orders)
    area = m.geometry()["area"]
    rng = np.random.default_rng(1)
    c = random_state(len(tri), orders, rng, mean_xi=0.0)
    c[0] = 0.0
    c[0, 0] = 0.5 * np.sqrt(area)
    u, st = m.usolve(O.Params(), c)
    assert st == 0
    assert np.abs(u - c[1:] / 3.0).max() < 1e-14 * np.abs(c[1:]).max()


def test_separation_identity():
    xy, tri, hv, orders = jittered_mixed(seed=8, pmin=1)
    m = O.Mesh(xy, tri, hv, orders)
    area = m.geometry()["area"]
    rng = np.random.default_rng(3)
    c = scale_state_means(random_state(len(tri), orders, rng), area)
    P = O.Params(g=9.81)
    full = m.rhs(P, c, part=0)
    base = m.rhs(P, c, part=1)
    corr = m.rhs(P, c, part=2)
    assert np.abs(base + corr - full).max() <= 1e-14 * np.abs(full).max()
    nb = m.neighbours()["nb"]
    lo = np.array([orders[e] <= 1 and all(n < 0 or orders[n] <= 1 for n in nb[e]) for e in range(len(tri))])
    assert lo.sum() > 0
    assert np.all(corr[:, :, lo] == 0.0)
    # base only ever touches modes of degree <= 1
    assert np.all(base[:, 3:, :] == 0.0)


def base_part_pin_error(Om):
    """relative error of the oracle's base part (Sect. 3: the terms whose test
    index and coefficient indices are all modes of degree <= 1) against its
    plain definition: the brute-force weak form of the state and of the
    scheme's own u with every mode of degree >= 2 set to zero, rows of degree
    <= 1, on tiny meshes with orders 0..4, an open-sea edge, friction and
    Coriolis; also the rows of degree >= 2, which the base part must leave zero"""
    worst = 0.0
    for case in range(3):
        xy, tri = tiny_meshes()[case]
        rng = np.random.default_rng(70 + case)
        ne = len(tri)
        orders = rng.integers(0, 5, size=ne).astype(np.int8)
        hv = 1.0 + 0.3 * rng.uniform(size=len(xy))
        bc, opened = None, []
        if case == 1:
            bc = np.zeros((ne, 3), np.int8)
            bc[0, 2] = 2
            opened = [(0, 2)]
        m = Om.Mesh(xy, tri, hv, orders, bc_tag=bc)
        geo = m.geometry()
        c = scale_state_means(random_state(ne, orders, rng), geo["area"])
        fr = dict(fric_lin=0.3, fric_quad=0.5, f_c=0.4)
        P = Om.Params(g=9.81, tide_amp=0.05, tide_period=0.0, **fr)
        _, u = m.rhs(P, c, t=0.0, with_u=True)
        base = m.rhs(P, c, t=0.0, part=1)
        ct, ut = c.copy(), u.copy()
        ct[:, 3:] = 0.0
        ut[:, 3:] = 0.0
        rb = dgref.brute_force_rhs(dgref.Tri(xy, tri), hv, orders, ct, ut, 9.81, bc_open=opened, xi_hat=0.05, **fr)
        scale = max(1.0, np.abs(rb[:, :3]).max())
        worst = max(worst, np.abs(base[:, :3] - rb[:, :3]).max() / scale, np.abs(base[:, 3:]).max() / scale)
    return worst


def tide_pin_error(Om):
    """relative difference between the oracle's rhs with the periodic open-sea
    elevation xi_hat(t) = amp sin(2 pi t / period + phase) at three times and
    its rhs with the constant elevation of that value (period 0), on a mesh
    with an open western side"""
    xy, tri, hv, orders = jittered_mixed(seed=12)
    bc = inputs.boundary_tags(xy, tri, "west")
    m = Om.Mesh(xy, tri, hv, orders, bc_tag=bc)
    rng = np.random.default_rng(12)
    c = scale_state_means(random_state(len(tri), orders, rng), m.geometry()["area"])
    amp, period, phase = 0.2, 700.0, 0.9
    worst = 0.0
    for t in (0.0, 130.0, 1234.5):
        r = m.rhs(Om.Params(g=9.81, tide_amp=amp, tide_period=period, tide_phase=phase), c, t=t)
        xh = amp * math.sin(2.0 * math.pi * t / period + phase)
        r0 = m.rhs(Om.Params(g=9.81, tide_amp=xh, tide_period=0.0), c, t=t)
        worst = max(worst, np.abs(r - r0).max() / np.abs(r0).max())
    return worst


def test_open_sea_elevation_is_the_tide_formula():
    assert tide_pin_error(O) <= 1e-13


def test_base_part_is_the_degree_one_truncation():
    assert base_part_pin_error(O) <= 1e-12


def test_rotation_equivariance():
    xy, tri, hv, orders = jittered_mixed(seed=9)
    rng = np.random.default_rng(4)
    m = O.Mesh(xy, tri, hv, orders)
    area = m.geometry()["area"]
    c = scale_state_means(random_state(len(tri), orders, rng), area)
    r = m.rhs(O.Params(g=9.81), c)
    xy2 = np.stack([-xy[:, 1], xy[:, 0]], axis=1)
    m2 = O.Mesh(xy2, tri, hv, orders)
    c2 = np.stack([c[0], -c[2], c[1]])
    r2 = m2.rhs(O.Params(g=9.81), c2)
    expect = np.stack([r[0], -r[2], r[1]])
    assert np.abs(r2 - expect).max() <= 1e-13 * np.abs(r).max()


def test_mass_conservation_walls():
    xy, tri, hv, orders = jittered_mixed(n=8, seed=10)
    m = O.Mesh(xy, tri, hv, orders)
    c = m.project_state(lambda x, y: (0.05 * np.exp(-((x - 0.4) ** 2 + (y - 0.6) ** 2) / 0.02), 0.0 * x, 0.0 * x))
    P = O.Params(g=9.81, rk_order=3, cfl=0.2)
    M0 = m.mass(c)
    area = m.geometry()["area"]
    Mref = M0 + np.sum(m.geometry()["hb"][:, 0] * np.sqrt(area))  # total water volume int H
    steps = 1000
    c1, t = m.run(P, c, 0.0, steps)
    assert t > 0
    assert abs(m.mass(c1) - M0) / Mref <= 1e-13 * math.sqrt(steps)
    assert np.abs(c1 - c).max() > 1e-6  # the state did evolve


def test_energy_matches_quadrature():
    xy, tri = tiny_meshes()[2]
    rng = np.random.default_rng(5)
    orders = rng.integers(0, 5, size=len(tri)).astype(np.int8)
    hv = 1.0 + 0.3 * rng.uniform(size=len(xy))
    m = O.Mesh(xy, tri, hv, orders)
    c = scale_state_means(random_state(len(tri), orders, rng), m.geometry()["area"])
    P = O.Params(g=2.0)
    E = m.energy(P, c)
    u, _ = m.usolve(P, c)
    msh = dgref.Tri(xy, tri)
    x, y, w = dgref.tri_rule(10)
    Eq = 0.0
    for e in range(len(tri)):
        K = K_OF_P[orders[e]]
        X, Y = msh.to_phys(e, x, y)
        ph, _, _ = msh.phys_basis(e, X, Y)
        f = lambda a: np.tensordot(a[:K], ph[:K], 1)  # noqa: E731
        Eq += np.sum(w * msh.det[e] * (0.5 * 2.0 * f(c[0, :, e]) ** 2 + 0.5 * (f(c[1, :, e]) * f(u[0, :, e]) + f(c[2, :, e]) * f(u[1, :, e]))))
    assert abs(E - Eq) <= 1e-13 * abs(Eq)


@pytest.mark.parametrize("rk,order", [(2, 2), (3, 3)])
def test_ssp_rk_temporal_order(rk, order):
    """Self-convergence in dt of the SSP-RK schemes (Sect. 2 time stepping)."""
    xy, tri = inputs.split_square_mesh(4, 1.0)
    hv = np.full(len(xy), 1.0)
    orders = np.full(len(tri), 2, np.int8)
    m = O.Mesh(xy, tri, hv, orders)
    c0 = m.project_state(lambda x, y: (0.05 * np.cos(math.pi * x) * np.cos(math.pi * y), 0.0 * x, 0.0 * x))
    P = O.Params(g=1.0, rk_order=rk)
    T_end = 0.08
    sols = []
    for nsteps in (8, 16, 32, 64):
        c, _ = m.run(P, c0, 0.0, nsteps, dt=T_end / nsteps)
        sols.append(c)
    e1 = np.abs(sols[0] - sols[3]).max()
    e2 = np.abs(sols[1] - sols[3]).max()
    e3 = np.abs(sols[2] - sols[3]).max()
    # errors against the finest run: e_k ~ C dt^order (1 - 2^-order(...)) -> ratio 2^order
    rate = math.log2((e1 - e2) / (e2 - e3))
    assert abs(rate - order) < 0.3, rate


def cfl_pin_error(Om):
    """relative error of the oracle's CFL step against its closed form on one
    right isosceles triangle with legs 2 (inscribed diameter 4|T|/perimeter)"""
    xy = np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 2.0]])
    tri = np.array([[0, 1, 2]])
    m = Om.Mesh(xy, tri, np.full(3, 4.0), np.array([1], np.int8))
    c = np.zeros((3, 15, 1))
    area = 2.0
    c[0, 0, 0] = 0.9 * math.sqrt(area)      # mean xi 0.9 -> H = 4.9
    c[1, 0, 0] = 4.9 * 3.0 * math.sqrt(area)  # u = 3
    c[2, 0, 0] = 4.9 * 4.0 * math.sqrt(area)  # v = 4
    P = Om.Params(g=10.0, cfl=0.5)
    d = 4 * area / (4 + 2 * math.sqrt(2))
    expect = 0.5 * d / ((5.0 + math.sqrt(49.0)) * 3)
    return abs(m.dt(P, c) - expect) / expect


def test_cfl_step_definition():
    assert cfl_pin_error(O) <= 1e-15


def indicator_pin_failures(Om):
    """the checks of the modal-decay indicator (the reading for the paper's
    dynamically p-adaptive runs, Sect. 2 end) against hand-computed energy
    fractions and decisions that the oracle `Om` fails (empty: none)"""
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    tri = np.array([[0, 1, 2], [1, 3, 2]])
    m = Om.Mesh(xy, tri, np.ones(4), np.array([2, 3], np.int8))
    c = np.zeros((3, 15, 2))
    # element 0, p = 2: degree-1 energy 2, degree-2 energy 0.03 -> s = 0.03 / 2.03
    c[0, :6, 0] = [5.0, 1.0, 1.0, 0.1, 0.1, 0.1]
    # element 1, p = 3: degree-3 modes zero -> s = 0
    c[0, :10, 1] = [3.0, 1.0, 0.5, 0.2, 0.0, 0.1, 0.0, 0.0, 0.0, 0.0]
    bad = []
    p, s, n = m.indicator(c, 0.01, 1e-4, 1, 4)
    if not (abs(s[0] - 0.03 / 2.03) < 1e-15 and s[1] == 0.0):
        bad.append("energy fractions")
    if not (list(p) == [3, 2] and n == 2):
        bad.append("decisions")
    p, s, n = m.indicator(c, 0.02, 1e-4, 1, 2)   # s[0] below theta_up; p_max caps nothing
    if not (list(p) == [2, 2] and n == 1):
        bad.append("theta_up")
    p, s, n = m.indicator(c, 0.01, 1e-4, 3, 4)   # p_min = 3 keeps element 1 at 3
    if list(p) != [3, 3]:
        bad.append("p_min")
    # hierarchical order change: dropped modes vanish, kept ones are untouched
    c2 = m.adapt_state(c, np.array([1, 3], np.int8))
    if not (np.all(c2[:, 3:, 0] == 0.0) and np.all(c2[:, :3, 0] == c[:, :3, 0]) and np.all(c2[:, :, 1] == c[:, :, 1])):
        bad.append("order change")
    return bad


def test_adaptivity_indicator_decisions():
    assert indicator_pin_failures(O) == []


def _dgref_modes(xy, tri, orders, f, nq=10):
    """c[3,15,ne] of f(x, y) -> (xi, U, V) by an independent quadrature with the
    scipy-evaluated basis (dgref), c_i = int_Omega_e f phi_{e,i} for i < K(p_e)"""
    msh = dgref.Tri(xy, tri)
    xh, yh, w = dgref.tri_rule(nq)
    c = np.zeros((3, 15, len(tri)))
    for e in range(len(tri)):
        K = K_OF_P[orders[e]]
        X, Y = msh.to_phys(e, xh, yh)
        ph, _, _ = msh.phys_basis(e, X, Y)
        for fld, val in enumerate(f(X, Y)):
            c[fld, :K, e] = (ph[:K] * (w * msh.det[e] * np.broadcast_to(val, X.shape))).sum(axis=1)
    return c


def mass_errors(Om, field):
    """relative errors of the mass of the oracle module Om (its own L2
    projection, then the independent quadrature) against the closed form"""
    xy, tri, hv, orders = jittered_mixed(n=6, seed=12)
    m = Om.Mesh(xy, tri, hv, orders)
    if field == "poly":
        f = lambda x, y: (1.0 + 2.0 * x - 3.0 * y * y + x * y * y, 0.0 * x, 0.0 * x)  # noqa: E731
        exact = 1.0 + 1.0 - 1.0 + 1.0 / 6.0
    else:
        f = lambda x, y: (np.sin(math.pi * x) * np.sin(math.pi * y), 0.0 * x, 0.0 * x)  # noqa: E731
        exact = 4.0 / math.pi ** 2
    area = m.geometry()["area"]
    assert area.max() / area.min() > 1.5  # a wrong per-element scale cannot hide
    return [abs(m.mass(c) - exact) / exact for c in (m.project_state(f, n=10), _dgref_modes(xy, tri, orders, f))]


MASS_TOL = {"poly": 1e-14, "sine": 1e-11}


@pytest.mark.parametrize("field", ["poly", "sine"])
def test_mass_is_the_integral_of_xi(field):
    """Mass (Sect. 2 diagnostics: int_Omega xi dx) equals the closed-form
    integral of the elevation over the unit square, on a jittered mesh whose
    element areas all differ and with orders 0..4.  A polynomial of degree 3
    is represented exactly by the modal coefficients' mean mode; the sine
    product's integral 4 / pi^2 is met to the quadrature error.  Two routes to
    the coefficients: the oracle's own L2 projection and an independent
    quadrature with the scipy-evaluated basis."""
    errs = mass_errors(O, field)
    assert max(errs) <= MASS_TOL[field], errs


def tide_order_rate(Om, rk):
    """observed temporal order of the oracle module Om under a time-dependent
    open-sea boundary (self-convergence, dt = T/10 .. T/80)"""
    xy, tri = inputs.split_square_mesh(4, 1.0)
    hv = np.full(len(xy), 1.0)
    orders = np.full(len(tri), 2, np.int8)
    bc = inputs.boundary_tags(xy, tri, "west")
    m = Om.Mesh(xy, tri, hv, orders, bc_tag=bc)
    c0 = np.zeros((3, 15, len(tri)))
    P = Om.Params(g=1.0, rk_order=rk, tide_amp=0.05, tide_period=0.4, tide_phase=0.3)
    T_end = 0.2
    sols = []
    for nsteps in (10, 20, 40, 80):
        c, t = m.run(P, c0, 0.0, nsteps, dt=T_end / nsteps)
        assert abs(t - T_end) < 1e-14
        sols.append(c)
    assert np.abs(sols[-1]).max() > 1e-3  # the tide moved the water
    e1 = np.abs(sols[0] - sols[3]).max()
    e2 = np.abs(sols[1] - sols[3]).max()
    e3 = np.abs(sols[2] - sols[3]).max()
    return math.log2((e1 - e2) / (e2 - e3))


@pytest.mark.parametrize("rk,order", [(2, 2), (3, 3)])
def test_ssp_rk_temporal_order_with_a_time_dependent_open_sea(rk, order):
    """Self-convergence in dt under a time-dependent open-sea boundary
    xi = xi_hat(t) (Sect. 2: the open-sea condition; SSP-RK time stepping):
    the boundary value enters every stage at its stage time t + tau_s dt, so
    the order holds only with the right stage times (0, 1 for the two-stage
    scheme; 0, 1, 1/2 for the three-stage one).  The tide swings through half
    a period in the run and drives the flow (the state starts at rest)."""
    rate = tide_order_rate(O, rk)
    assert abs(rate - order) < 0.3, rate


def _evaluate(xy, tri, c_f, orders, pts_per_elem=7, seed=0):
    """the modal field c_f[15, ne] at random points of every element, with the
    scipy-evaluated basis (dgref); returns (points x, y, values)"""
    msh = dgref.Tri(xy, tri)
    rng = np.random.default_rng(seed)
    X, Y, F = [], [], []
    for e in range(len(tri)):
        a, b = rng.uniform(size=(2, pts_per_elem))
        flip = a + b > 1.0
        a[flip], b[flip] = 1.0 - a[flip], 1.0 - b[flip]
        x, y = msh.to_phys(e, a, b)
        ph, _, _ = msh.phys_basis(e, x, y)
        K = K_OF_P[orders[e]]
        X.append(x); Y.append(y); F.append(np.tensordot(c_f[:K, e], ph[:K], 1))
    return np.concatenate(X), np.concatenate(Y), np.concatenate(F)


def test_projection_reproduces_polynomials_of_the_element_order():
    """The oracle's L2 projection (the initial-state route of the tests) is
    exact on polynomials of degree <= p_e: evaluated with the independent
    basis, the projected field equals the polynomial pointwise."""
    xy, tri, hv, orders = jittered_mixed(n=4, seed=13, pmin=2, pmax=4)
    m = O.Mesh(xy, tri, hv, orders)
    f = lambda x, y: (0.3 - 0.2 * x + 0.5 * y + 0.7 * x * y - 0.4 * y * y, 0.0 * x, 0.0 * x)  # noqa: E731
    c = m.project_state(f, n=8)
    x, y, val = _evaluate(xy, tri, c[0], orders)
    assert np.abs(val - f(x, y)[0]).max() <= 1e-13


def test_p1_modes_reproduce_the_vertex_interpolant():
    """or_p1_modes (vertex values -> modes 1..3, the bathymetry's and the
    benchmarks' initial states' route) reproduces the continuous piecewise-
    linear interpolant: exact for a linear function, and equal to the vertex
    values at the vertices of every element for arbitrary ones."""
    xy, tri, hv, orders = jittered_mixed(n=5, seed=14)
    m = O.Mesh(xy, tri, hv, np.ones(len(tri), np.int8))
    lin = 0.4 + 1.3 * xy[:, 0] - 0.7 * xy[:, 1]
    c = np.zeros((15, len(tri)))
    c[:3] = m.p1_modes(lin)
    x, y, val = _evaluate(xy, tri, c, np.ones(len(tri), np.int8))
    assert np.abs(val - (0.4 + 1.3 * x - 0.7 * y)).max() <= 1e-13
    rnd = np.random.default_rng(3).standard_normal(len(xy))
    c[:3] = m.p1_modes(rnd)
    msh = dgref.Tri(xy, tri)
    for e in range(len(tri)):
        vx, vy = xy[msh.tri[e], 0], xy[msh.tri[e], 1]
        ph, _, _ = msh.phys_basis(e, vx - 1e-12 * (vx - vx.mean()), vy - 1e-12 * (vy - vy.mean()))
        assert np.abs(np.tensordot(c[:3, e], ph[:3], 1) - rnd[msh.tri[e]]).max() <= 1e-9


def test_threaded_oracle_is_bitwise_the_serial_one():
    """The threaded build (OpenMP over elements; the bench's all-core baseline
    and the long parity runs use it) gives bitwise the serial results: the
    projection, 5 CFL steps with an open-sea tide and the indicator."""
    xy, tri, hv, orders = jittered_mixed(n=10, seed=15, pmin=0, pmax=4)
    bc = inputs.boundary_tags(xy, tri, "west")
    ic = lambda x, y: (0.1 * np.exp(-((x - 0.4) ** 2 + (y - 0.6) ** 2) / 0.02), 0.05 + 0.0 * x, 0.0 * x)  # noqa: E731
    P = O.Params(g=9.81, rk_order=3, cfl=0.2, tide_amp=0.02, tide_period=0.5)
    out = []
    for threads in (1, 4):
        m = O.Mesh(xy, tri, hv, orders, bc_tag=bc, threads=threads)
        c = m.project_state(ic)
        c5, t5 = m.run(P, c, 0.0, 5)
        out.append((c, c5, t5, m.indicator(c5, 0.05, 1e-3, 0, 4)[0]))
    assert O.threaded(4) == 4
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
