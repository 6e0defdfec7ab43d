"""CUDA path against the FP64 oracle, through the C ABI (needs a GB300).

Tolerances: the FP64 path must match the oracle to 1e-11 relative L2 after
1000 steps (same seeded inputs); one rhs evaluation agrees to ~1e-13 (only
the summation order and the tensors' last bits differ).  The mixed mode
(FP32 correction) must stay within 1e-6 relative L2.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2311_11348_gb300 import build, inputs, swedg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    swedg.load()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_pair(w, precision=swedg.PREC_FP64, tide=(0.0, 0.0, 0.0), rk=None, cfl=None):
    m = O.Mesh(w["xy"], w["tri"], w["hv"], w["orders"], bc_tag=w.get("bc_tag"))
    P = O.Params(g=w["g"], cfl=cfl or w["cfl"], rk_order=rk or w["rk_order"], tide_amp=tide[0], tide_period=tide[1],
                 tide_phase=tide[2])
    s = swedg.Solver(g=w["g"], cfl=cfl or w["cfl"], rk_order=rk or w["rk_order"], precision=precision, tide=tide)
    s.set_mesh(w["xy"], w["tri"], w.get("bc_tag"))
    s.set_bathymetry(w["hv"])
    s.set_orders(w["orders"])
    return m, P, s


def mixed_workload(n=16, seed=1, pmin=0, pmax=4, open_west=True):
    xy, tri = inputs.split_square_mesh(n, 1e4, jitter=0.2, seed=seed)
    rng = np.random.default_rng(seed)
    hv = inputs.fourier_bathymetry(xy, 1e4, lo=20.0, hi=200.0, seed=seed + 1)
    orders = rng.integers(pmin, pmax + 1, size=len(tri)).astype(np.int8)
    bc = inputs.boundary_tags(xy, tri, "west") if open_west else None

    def ic(x, y):
        return 0.5 * np.exp(-((x - 6e3) ** 2 + (y - 4e3) ** 2) / 2e6), 3.0 * np.exp(-((x - 5e3) ** 2) / 4e6), \
            -2.0 * np.exp(-((y - 5e3) ** 2) / 5e6)

    return dict(xy=xy, tri=tri, hv=hv, orders=orders, ic=ic, bc_tag=bc, g=9.81, rk_order=3, cfl=0.2)


def test_rhs_unit_p1():
    w = inputs.unit_p1()
    m, P, s = make_pair(w)
    c = m.project_state(w["ic"])
    r_o = m.rhs(P, c)
    r_g = s.rhs(c)
    assert rel_l2(r_g, r_o) < 1e-13
    assert np.abs(r_g - r_o).max() <= 1e-12 * np.abs(r_o).max()


@pytest.mark.parametrize("seed", [1, 2])
def test_rhs_mixed_orders_open_sea(seed):
    w = mixed_workload(seed=seed)
    tide = (0.3, 3600.0, 0.4)
    m, P, s = make_pair(w, tide=tide)
    c = m.project_state(w["ic"])
    t0 = 500.0
    s.set_state(c, t0)
    r_o = m.rhs(P, c, t=t0)
    r_g = s.rhs(c)
    assert np.abs(r_g - r_o).max() <= 1e-12 * np.abs(r_o).max()
    b_g, k_g = s.rhs_parts(c)
    b_o = m.rhs(P, c, t=t0, part=1)
    k_o = m.rhs(P, c, t=t0, part=2)
    assert np.abs(b_g - b_o).max() <= 1e-12 * np.abs(b_o).max()
    assert np.abs(k_g - k_o).max() <= 1e-12 * np.abs(r_o).max()
    assert np.abs(b_g + k_g - r_g).max() <= 1e-13 * np.abs(r_o).max()


def test_single_triangle_and_p0():
    xy = np.array([[0.0, 0.0], [2.0, 0.3], [0.5, 1.7]])
    tri = np.array([[0, 2, 1]], dtype=np.int32)  # clockwise on purpose
    for p in range(5):
        w = dict(xy=xy, tri=tri, hv=np.array([1.0, 1.5, 2.0]), orders=np.array([p], np.int8), g=9.81, rk_order=2,
                 cfl=0.1)
        m, P, s = make_pair(w)
        c = m.project_state(lambda x, y: (0.1 * x * y, 0.2 + 0.1 * x, -0.1 * y))
        assert np.abs(s.rhs(c) - m.rhs(P, c)).max() <= 1e-12 * max(1.0, np.abs(m.rhs(P, c)).max())


def test_fp64_1000_steps_unit_p1():
    """The FP64 gate: 1000 CFL steps of SSP-RK2 on the 512-triangle p = 1 case."""
    w = inputs.unit_p1()
    m, P, s = make_pair(w)
    c = m.project_state(w["ic"])
    s.set_state(c, 0.0)
    t_g = s.run(1000)
    c_g, _ = s.get_state()
    c_o, t_o = m.run(P, c, 0.0, 1000)
    assert abs(t_g - t_o) <= 1e-12 * t_o
    assert rel_l2(c_g, c_o) < 1e-11
    assert abs(s.mass() - m.mass(c_o)) <= 1e-12 * abs(m.mass(c_o))


def test_fp64_steps_mixed_orders():
    w = mixed_workload(seed=3, pmin=1, pmax=4)
    m, P, s = make_pair(w, tide=(0.2, 2000.0, 0.0))
    c = m.project_state(w["ic"])
    s.set_state(c, 0.0)
    n = 200
    s.run(n)
    c_g, t_g = s.get_state()
    c_o, t_o = m.run(P, c, 0.0, n)
    assert abs(t_g - t_o) <= 1e-12 * t_o
    assert rel_l2(c_g, c_o) < 1e-11


def test_mixed_fp32_correction_accuracy():
    w = mixed_workload(seed=4, pmin=1, pmax=3, open_west=False)
    m, P, s = make_pair(w, precision=swedg.PREC_MIXED_FP32)
    c = m.project_state(w["ic"])
    s.set_state(c, 0.0)
    n = 200
    s.run(n, dt_fixed=0.5)
    c_g, _ = s.get_state()
    c_o, _ = m.run(P, c, 0.0, n, dt=0.5)
    err = rel_l2(c_g, c_o)
    assert err < 1e-6, err
    # the base modes carry the mass, and the correction's share of the mean mode
    # is accumulated in FP64 from one flux value per edge: conserved to FP64
    # round-off even with an FP32 correction
    m0 = m.mass(c)
    assert abs(s.mass() - m0) <= 1e-13 * math.sqrt(n) * abs(m0)


@pytest.mark.parametrize("p", [0, 2, 4])
@pytest.mark.parametrize("precision", [swedg.PREC_FP64, swedg.PREC_MIXED_FP32, swedg.PREC_MIXED_TF32])
def test_uniform_order_meshes(precision, p):
    """one order everywhere (288 triangles, a ragged tail of every 128-wide
    launch): p = 0 leaves the correction branch without elements, p = 4 the
    base branch without base-only elements; 20 CFL steps of SSP-RK3 with the
    tide on the open western side against the oracle (relative L2 1e-11 in
    FP64, 1e-6 with the FP32 or tensor-core correction)"""
    w = mixed_workload(n=12, seed=7, pmin=p, pmax=p)
    tide = (0.2, 1800.0, 0.3)
    m, P, s = make_pair(w, precision=precision, tide=tide)
    c = m.project_state(w["ic"])
    s.set_state(c, 0.0)
    t_g = s.run(20)
    c_g, _ = s.get_state()
    c_o, t_o = m.run(P, c, 0.0, 20)
    tol = 1e-11 if precision == swedg.PREC_FP64 else 1e-6
    assert rel_l2(c_g, c_o) < tol, rel_l2(c_g, c_o)
    assert abs(t_g - t_o) <= tol * t_o
    s.close()


@pytest.mark.parametrize("precision", [swedg.PREC_MIXED_FP32, swedg.PREC_MIXED_TF32])
def test_mixed_rhs_of_the_higher_modes_over_deep_water(precision):
    """The bottom term g xi h_b of the higher test modes (h_b of 50..4000 m
    against xi of 1 m): the correction kernels carry its degree-1 part as g h_b
    times the FP64 jump of the degree-1 elevation instead of a volume and an
    edge integral that cancel in FP32.  One rhs of the 64x64 ocean recipe after
    50 oracle steps: the higher momentum modes within 2e-7 of the oracle's
    (relative to the rhs norm; measured 2.9e-8; with the two integrals formed
    separately in FP32 the same modes were off by about 3e-6)"""
    w = inputs.ocean_p123(64)
    m = O.Mesh(w["xy"], w["tri"], w["hv"], w["orders"], threads=0)
    P = O.Params(g=9.81, cfl=0.1, rk_order=3)
    c0 = np.zeros((3, 15, len(w["tri"])))
    c0[0, :3] = m.p1_modes(w["ic"](w["xy"][:, 0], w["xy"][:, 1])[0])
    c, _ = m.run(P, c0, 0.0, 50)
    r_o = m.rhs(P, c)
    s = swedg.Solver(g=9.81, cfl=0.1, rk_order=3, precision=precision)
    s.set_mesh(w["xy"], w["tri"])
    s.set_bathymetry(w["hv"])
    s.set_orders(w["orders"])
    d = s.rhs(c) - r_o
    s.close()
    nr = np.linalg.norm(r_o)
    assert np.linalg.norm(d[1, 3:]) / nr < 2e-7
    assert np.linalg.norm(d[2, 3:]) / nr < 2e-7
    assert np.linalg.norm(d) / nr < 2e-7


@pytest.mark.parametrize("precision", [swedg.PREC_FP64, swedg.PREC_MIXED_FP32, swedg.PREC_MIXED_TF32])
def test_friction_and_coriolis(precision):
    """Bottom friction (tau from the element means, Sect. 3) and Coriolis of
    Eq. (5): one rhs with inflated coefficients (so that the source terms are a
    visible part of it) and 100 CFL steps with the paper's tidal-setup values."""
    w = mixed_workload(seed=8, pmin=0, pmax=4)
    big = dict(fric_lin=0.05, fric_quad=0.5, f_c=0.02)
    m = O.Mesh(w["xy"], w["tri"], w["hv"], w["orders"], bc_tag=w["bc_tag"])
    c = m.project_state(w["ic"])
    s = swedg.Solver(g=w["g"], cfl=w["cfl"], rk_order=3, precision=precision,
                     friction=(big["fric_lin"], big["fric_quad"]), f_c=big["f_c"])
    s.set_mesh(w["xy"], w["tri"], w["bc_tag"])
    s.set_bathymetry(w["hv"])
    s.set_orders(w["orders"])
    s.set_state(c, 0.0)
    r_o = m.rhs(O.Params(g=w["g"], **big), c)
    r_0 = m.rhs(O.Params(g=w["g"]), c)
    assert np.abs(r_o - r_0).max() > 1e-3 * np.abs(r_o).max()
    r_g = s.rhs(c)
    tol = 1e-12 if precision == swedg.PREC_FP64 else 5e-6
    assert rel_l2(r_g, r_o) < tol, rel_l2(r_g, r_o)
    s.close()
    real = dict(fric_lin=0.0, fric_quad=0.009, f_c=3.19e-5)
    s = swedg.Solver(g=w["g"], cfl=w["cfl"], rk_order=3, precision=precision,
                     friction=(real["fric_lin"], real["fric_quad"]), f_c=real["f_c"])
    s.set_mesh(w["xy"], w["tri"], w["bc_tag"])
    s.set_bathymetry(w["hv"])
    s.set_orders(w["orders"])
    s.set_state(c, 0.0)
    s.run(100)
    c_g, t_g = s.get_state()
    P = O.Params(g=w["g"], cfl=w["cfl"], rk_order=3, **real)
    c_o, t_o = m.run(P, c, 0.0, 100)
    err = rel_l2(c_g, c_o)
    print("friction + Coriolis, 100 steps, precision", precision, "rel L2", err)
    assert err < (1e-11 if precision == swedg.PREC_FP64 else 1e-6), err
    s.close()


def test_full_size_ocean_rhs():
    """Full-size workload (131,072 triangles, p in {1,2,3}): one rhs, all outputs."""
    w = inputs.ocean_p123()
    m, P, s = make_pair(w)
    c = m.project_state(w["ic"], n=6)
    r_o = m.rhs(P, c)
    r_g = s.rhs(c)
    assert np.abs(r_g - r_o).max() <= 1e-12 * np.abs(r_o).max()


def test_lake_at_rest_and_mass_gpu():
    w = mixed_workload(seed=5, pmin=0, pmax=4, open_west=False)
    m, P, s = make_pair(w)
    area = m.geometry()["area"]
    c = np.zeros((3, 15, len(w["tri"])))
    c[0, 0] = 0.37 * np.sqrt(area)
    s.set_state(c, 0.0)
    s.run(50)
    c1, _ = s.get_state()
    assert np.abs(c1 - c).max() <= 1e-12 * np.abs(c).max()
    c = m.project_state(w["ic"])
    s.set_state(c, 0.0)
    m0 = s.mass()
    s.run(100)
    Mref = np.sum((m.geometry()["hb"][:, 0] + c[0, 0]) * np.sqrt(area))
    assert abs(s.mass() - m0) <= 1e-13 * math.sqrt(100) * Mref


def test_checkpoint_resume_is_bitwise():
    w = mixed_workload(seed=6, pmin=1, pmax=3, open_west=False)
    m, P, s = make_pair(w)
    c = m.project_state(w["ic"])
    s.set_state(c, 0.0)
    s.run(20)
    ref, tref = s.get_state()
    s.set_state(c, 0.0)
    s.run(10)
    mid, tmid = s.get_state()
    _, _, s2 = make_pair(w)
    s2.set_state(mid, tmid)
    s2.run(10)
    out, tout = s2.get_state()
    assert tout == tref
    assert np.array_equal(out, ref)


def pack(c, orders):
    """the packed layout written out from the full one: element by element, xi, U, V modes < K(p)"""
    return np.concatenate([c[:, :(p + 1) * (p + 2) // 2, u].ravel() for u, p in enumerate(orders)])


@pytest.mark.parametrize("precision", [swedg.PREC_FP64, swedg.PREC_MIXED_FP32])
def test_packed_state_round_trip_and_steps(precision):
    """the packed state calls move exactly the modes each order has; a run fed
    through them is bitwise the run fed through the full layout"""
    import torch
    w = mixed_workload(seed=7, pmin=0, pmax=4)
    m, P, s = make_pair(w, precision)
    c = m.project_state(w["ic"])
    K = np.array([(p + 1) * (p + 2) // 2 for p in w["orders"]])
    assert s.packed_size() == 3 * K.sum()
    s.set_state(c, 0.0)
    s.run(3)
    full, t = s.get_state()
    packed, tp = s.get_state_packed()
    assert tp == t and np.array_equal(packed, pack(full, w["orders"]))
    dev = torch.from_numpy(packed).cuda()  # device buffers too
    back = torch.zeros_like(dev)
    _, _, s2 = make_pair(w, precision)
    s2.set_state_packed(dev, t)
    s2.get_state_packed(back)
    assert torch.equal(back, dev)
    s.run(5)
    s2.run(5)
    assert np.array_equal(s2.get_state()[0], s.get_state()[0])
    with pytest.raises(ValueError):
        s2.set_state_packed(packed[:-1], 0.0)


def test_errors_are_reported_not_faulted():
    w = inputs.unit_p1()
    _, _, s = make_pair(w)
    with pytest.raises(swedg.SweError) as ei:
        s.set_orders(np.full(len(w["tri"]), 7, np.int8))
    assert ei.value.code == -1
    bad = w["tri"].copy()
    bad[0] = [0, 0, 1]
    with pytest.raises(swedg.SweError) as ei:
        s.set_mesh(w["xy"], bad)
    assert ei.value.code == -2
    # an empty mesh and a boundary tag outside 0..2 are invalid arguments;
    # after a failed set_mesh the context holds no mesh
    with pytest.raises(swedg.SweError) as ei:
        s.set_mesh(w["xy"], np.zeros((0, 3), np.int32))
    assert ei.value.code == -1
    tags = np.zeros((len(w["tri"]), 3), np.int8)
    tags[len(tags) // 2, 1] = 3
    with pytest.raises(swedg.SweError) as ei:
        s.set_mesh(w["xy"], w["tri"], tags)
    assert ei.value.code == -1 and "boundary tag" in str(ei.value)
    with pytest.raises(swedg.SweError) as ei:
        s.set_state(np.zeros((3, 15, len(w["tri"]))), 0.0)
    assert ei.value.code == -1
    s.set_mesh(w["xy"], w["tri"])
    s.set_bathymetry(np.full(len(w["xy"]), 1.0))
    c = np.zeros((3, 15, len(w["tri"])))
    c[0, 0] = -5.0  # xi = -5 on a 1 m deep basin
    s.set_state(c, 0.0)
    with pytest.raises(swedg.SweError) as ei:
        s.rk_step(1e-3)
    assert ei.value.code in (-3, -4)


def test_non_manifold_mesh_is_rejected():
    """three triangles on the edge (1, 2): the adjacency build reports it"""
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0], [0.5, -1.0]])
    tri = np.array([[0, 1, 2], [1, 3, 2], [1, 2, 4]], np.int32)
    s = swedg.Solver(g=9.81, cfl=0.2, rk_order=3)
    with pytest.raises(swedg.SweError) as ei:
        s.set_mesh(xy, tri)
    assert ei.value.code == -2 and "more than 2" in str(ei.value)
    s.set_mesh(xy, tri[:2])
    s.close()


def test_renumbered_mesh_matches_the_oracle():
    """vertex ids and triangles in random order (no locality in the edge
    buckets): the right-hand side still equals the oracle's on that mesh"""
    w = mixed_workload(n=20, seed=3)
    rng = np.random.default_rng(5)
    pv = rng.permutation(len(w["xy"]))
    inv = np.argsort(pv)
    pt = rng.permutation(len(w["tri"]))
    w = dict(w, xy=w["xy"][pv], hv=w["hv"][pv], tri=inv[w["tri"][pt]].astype(np.int32), orders=w["orders"][pt],
             bc_tag=w["bc_tag"][pt])
    m, P, s = make_pair(w)
    c = m.project_state(w["ic"])
    r_o = m.rhs(P, c)
    r_g = s.rhs(c)
    assert np.abs(r_g - r_o).max() <= 1e-12 * np.abs(r_o).max()
    s.close()


def test_device_wait_timeout_is_reported_and_the_context_survives():
    """The failure path of the bounded device waits, without a GPU fault: a
    wait that nothing completes runs out, the call returns SWE_ETIMEOUT, and
    the same context then steps exactly like a fresh one."""
    w = mixed_workload(seed=9, pmin=1, pmax=4)
    m, P, s = make_pair(w, precision=swedg.PREC_MIXED_TF32)
    c = m.project_state(w["ic"])
    s.set_state(c, 0.0)
    with pytest.raises(swedg.SweError) as ei:
        s.selftest_wait(1000)
    assert ei.value.code == -6
    s.run(5)
    a, _ = s.get_state()
    _, _, f = make_pair(w, precision=swedg.PREC_MIXED_TF32)
    f.set_state(c, 0.0)
    f.run(5)
    b, _ = f.get_state()
    assert np.array_equal(a, b)
    s.close()
    f.close()


def test_full_size_shelf_rhs_p1234_open_sea():
    """The paper's mesh size (2,097,152 triangles) with p in {1..4} and the M2
    open-sea boundary on x = 0: one rhs, all outputs, against the oracle."""
    w = inputs.shelf_p1234()
    amp, period, phase = w["tide"]
    tide = (amp, period, phase)
    m, P, s = make_pair(w, tide=tide)
    # P1 interpolants of smooth fields plus seeded higher modes (a full L2
    # projection at this size takes minutes in the oracle)
    x, y = w["xy"][:, 0], w["xy"][:, 1]
    ne = len(w["tri"])
    c = np.zeros((3, 15, ne))
    c[0, :3] = m.p1_modes(w["ic"](x, y)[0])
    c[1, :3] = m.p1_modes(50.0 * np.sin(2 * np.pi * y / 5e5))
    c[2, :3] = m.p1_modes(-30.0 * np.cos(2 * np.pi * x / 5e5))
    rng = np.random.default_rng(12)
    K = np.array([1, 3, 6, 10, 15])[w["orders"]]
    scale = np.abs(c[:, :3]).max(axis=(1, 2))
    for f in range(3):
        hi = rng.standard_normal((12, ne)) * 1e-3 * scale[f]
        c[f, 3:] = np.where(np.arange(3, 15)[:, None] < K[None, :], hi, 0.0)
    t0 = 3600.0
    s.set_state(c, t0)
    r_o = m.rhs(P, c, t=t0)
    r_g = s.rhs(c)
    assert np.abs(r_g - r_o).max() <= 1e-12 * np.abs(r_o).max()
    s.close()


@pytest.mark.parametrize("precision", [swedg.PREC_MIXED_FP32, swedg.PREC_MIXED_TF32])
def test_dynamic_adaptivity_mixed_modes(precision):
    """swe_run_adaptive in the mixed modes: the same order decisions as the FP64
    oracle (no indicator value within 1e-5 of a threshold, far above the mixed
    modes' error) and the state within 1e-6."""
    w = mixed_workload(seed=7, pmin=1, pmax=2, open_west=False)
    up, down, pmin, pmax = 5e-2, 1e-3, 1, 4
    m, P, s = make_pair(w, precision=precision)
    c = m.project_state(w["ic"])
    s.set_state(c, 0.0)
    dt = 0.25
    co = c.copy()
    for rnd in range(3):
        co, _ = m.run(P, co, 0.0, 10, dt=dt)
        new, sv, n = m.indicator(co, up, down, pmin, pmax)
        for th in (up, down):
            assert np.all(np.abs(sv - th) > 1e-5 * th)
        co = m.adapt_state(co, new)
    s.run_adaptive(30, 10, up, down, pmin, pmax, dt_fixed=dt)
    cg, _ = s.get_state()
    err = rel_l2(cg, co)
    print("adaptive, precision", precision, "rel L2", err, "orders", np.bincount(new, minlength=5))
    assert err < 1e-6, err
    po, _, _ = m.indicator(co, up, down, pmin, pmax)
    o2, _ = s.adapt(up, down, pmin, pmax)
    assert np.array_equal(o2, po)
    s.close()


def test_dynamic_adaptivity_matches_oracle():
    """swe_run_adaptive (indicator every 10 steps, hierarchical order changes)
    against the oracle doing the same: orders bit-exact, state to 1e-11."""
    w = mixed_workload(seed=7, pmin=1, pmax=2, open_west=False)
    up, down, pmin, pmax = 5e-2, 1e-3, 1, 3
    m, P, s = make_pair(w)
    c = m.project_state(w["ic"])
    s.set_state(c, 0.0)
    dt = 0.5
    orders = w["orders"].copy()
    co = c.copy()
    nchanged = []
    for rnd in range(3):
        co, _ = m.run(P, co, 0.0, 10, dt=dt)
        new, sv, n = m.indicator(co, up, down, pmin, pmax)
        # no indicator value within round-off of a threshold (the decision would be ambiguous)
        for th in (up, down):
            assert np.all(np.abs(sv - th) > 1e-9 * th)
        co = m.adapt_state(co, new)
        orders = new
        nchanged.append(n)
    assert min(nchanged) > 0 and len(set(orders)) == 3
    s.run_adaptive(30, 10, up, down, pmin, pmax, dt_fixed=dt)
    cg, _ = s.get_state()
    assert rel_l2(cg, co) < 1e-11
    # the library's current orders equal the oracle's
    _, nchg = s.adapt(1e300, -1.0, pmin, pmax)  # thresholds that change nothing
    assert nchg == 0
    o2, _ = s.adapt(up, down, pmin, pmax)
    po, _, _ = m.indicator(co, up, down, pmin, pmax)
    assert np.array_equal(o2, po)


@pytest.mark.parametrize("precision", [swedg.PREC_FP64, swedg.PREC_MIXED_FP32])
def test_base_work_schedules_give_the_same_state(precision):
    """Static grid-stride shares and dynamic tiles of 1, 3 and 16 x base
    threads units (ticket counters that every launch leaves at zero for the
    next one: 30 graph replays of 3 stages, then an rhs) give bitwise the same
    state, the oracle's to 1e-11 in FP64"""
    w = mixed_workload(n=20, seed=5, pmin=1, pmax=4)
    m, P, _ = make_pair(w)
    c = m.project_state(w["ic"])
    got = []
    for shape in ((1, 64, 256, 128, 0, 0), (1, 64, 256, 128, 0, 1), (3, 128, 256, 128, 1, 3), (1, 32, 256, 64, 0, 16)):
        _, _, s = make_pair(w, precision=precision)
        s.set_launch_shape(shape)
        s.set_state(c, 0.0)
        s.run(30)
        cg, t = s.get_state()
        got.append((cg, t, s.rhs(cg)))
        s.close()
    for g in got[1:]:
        assert g[1] == got[0][1]
        assert np.array_equal(g[0], got[0][0]) and np.array_equal(g[2], got[0][2])
    if precision == swedg.PREC_FP64:
        co, to = m.run(P, c, 0.0, 30)
        assert rel_l2(got[0][0], co) < 1e-11 and abs(got[0][1] - to) <= 1e-12 * to


@pytest.mark.parametrize("precision", [swedg.PREC_FP64, swedg.PREC_MIXED_FP32])
def test_async_packed_pipeline_equals_the_synchronous_calls(precision):
    """swe_set_state_packed_async / swe_run_async / swe_get_state_packed_async
    with pinned host buffers, six different inputs in a row and one swe_sync
    at the end (copies double-buffered on their own streams): every output is
    bitwise the synchronous calls' result; a state with a negative depth
    enqueued the same way is reported by swe_sync"""
    import torch
    w = mixed_workload(n=18, seed=6, pmin=1, pmax=4)
    m, P, s = make_pair(w, precision=precision)
    base = m.project_state(w["ic"])
    n = s.packed_size()
    ins, refs = [], []
    for k in range(6):
        c = base.copy()
        c[1:] *= 1.0 + 0.1 * k
        s.set_state(c, 0.0)
        packed, _ = s.get_state_packed()
        ins.append(torch.from_numpy(packed).pin_memory())
        s.set_state_packed(packed, 10.0 * k)
        s.run(2)
        refs.append(s.get_state_packed()[0])
    outs = [torch.zeros(n, dtype=torch.float64).pin_memory() for _ in range(6)]
    for k in range(6):
        s.set_state_packed_async(ins[k], 10.0 * k)
        s.run_async(2)
        s.get_state_packed_async(outs[k])
    s.sync()
    for k in range(6):
        assert np.array_equal(outs[k].numpy(), refs[k]), k
    bad = ins[0].clone()
    bad_c = base.copy()
    bad_c[0, 0] = -1e4 * np.sqrt(m.geometry()["area"])
    s.set_state(bad_c, 0.0)
    bad.copy_(torch.from_numpy(s.get_state_packed()[0]))
    s.set_state_packed_async(bad, 0.0)
    s.run_async(1)
    with pytest.raises(swedg.SweError) as ei:
        s.sync()
    assert ei.value.code in (-3, -4)
    s.close()


@pytest.mark.parametrize("precision", [swedg.PREC_FP64, swedg.PREC_MIXED_FP32, swedg.PREC_MIXED_TF32])
def test_order_change_on_the_device_equals_a_fresh_build(precision):
    """swe_set_orders on a built context regroups the elements on the device
    (stable partition by order, correction edges, packed offsets) and carries
    the state over hierarchically: the steps that follow are bitwise those of
    a context built afresh with the new orders from the truncated state, and
    the footprint is at least the fresh build's"""
    from paper_2311_11348_gb300 import serve
    w = mixed_workload(n=14, seed=8, pmin=0, pmax=4)
    m, P, s = make_pair(w, precision=precision)
    c = m.project_state(w["ic"])
    s.set_state(c, 0.0)
    s.run(5)
    c5, t5 = s.get_state()
    new = np.random.default_rng(9).integers(0, 5, size=len(w["tri"])).astype(np.int8)
    s.set_orders(new)
    got_c, _ = s.get_state()
    K = np.array([1, 3, 6, 10, 15])[new]
    assert np.array_equal(got_c, np.where(np.arange(15)[None, :, None] < K[None, None, :], c5, 0.0))
    s.run(5)
    got, tg = s.get_state()
    w2 = dict(w, orders=new)
    _, _, f = make_pair(w2, precision=precision)
    f.set_state(c5, t5)
    f.run(5)
    ref, tr = f.get_state()
    assert tg == tr and np.array_equal(got, ref)
    assert s.memory_bytes() >= f.memory_bytes() == serve.device_bytes([w2], precision)
    assert s.packed_size() == f.packed_size()
    s.close()
    f.close()
