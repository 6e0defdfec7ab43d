"""Tensor-core correction mode (SWE_PREC_MIXED_TF32) against the FP64 oracle,
through the C ABI (needs a GB300).

The momentum volume terms of the higher modes run as TF32 head/tail GEMMs
with FP32 accumulation (about 21 bits), everything else as in the FP32
correction mode, so the state bounds are those of that mode: 1e-6 relative
L2 after 200 steps, mass to FP64 round-off (the base modes stay FP64).  A
single right-hand side is held to 5e-6 relative L2 (1e-5 on the rows of the
higher modes, which are sums with cancellation): the tensor cores' FP32
accumulation is measurably less exact than FP32 FMA chains (1.5-3e-6 against
0.5-1.4e-6 of the FP32 correction on these meshes).  The meshes give every
order group a ragged last tile of 128 elements."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2311_11348_gb300 import build, inputs, serve, swedg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    swedg.load()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def workload(n, seed, pmin=1, pmax=4, open_west=True):
    xy, tri = inputs.split_square_mesh(n, 1e4, jitter=0.2, seed=seed)
    rng = np.random.default_rng(seed)
    hv = inputs.fourier_bathymetry(xy, 1e4, lo=20.0, hi=200.0, seed=seed + 1)
    orders = rng.integers(pmin, pmax + 1, size=len(tri)).astype(np.int8)
    bc = inputs.boundary_tags(xy, tri, "west") if open_west else None

    def ic(x, y):
        return 0.5 * np.exp(-((x - 6e3) ** 2 + (y - 4e3) ** 2) / 2e6), 3.0 * np.exp(-((x - 5e3) ** 2) / 4e6), \
            -2.0 * np.exp(-((y - 5e3) ** 2) / 5e6)

    return dict(xy=xy, tri=tri, hv=hv, orders=orders, ic=ic, bc_tag=bc, g=9.81, rk_order=3, cfl=0.2)


def solver(w, precision, tide=(0.0, 0.0, 0.0)):
    s = swedg.Solver(g=w["g"], cfl=w["cfl"], rk_order=w["rk_order"], precision=precision, tide=tide)
    s.set_mesh(w["xy"], w["tri"], w.get("bc_tag"))
    s.set_bathymetry(w["hv"])
    s.set_orders(w["orders"])
    return s


@pytest.mark.parametrize("n,seed", [(13, 1), (40, 2)])
def test_tc_rhs_matches_oracle(n, seed):
    w = workload(n, seed)
    counts = np.bincount(w["orders"], minlength=5)
    assert all(c % 128 for c in counts[2:])  # ragged last tiles
    m = O.Mesh(w["xy"], w["tri"], w["hv"], w["orders"], bc_tag=w["bc_tag"])
    tide = (0.3, 3600.0, 0.4)
    P = O.Params(g=w["g"], cfl=w["cfl"], rk_order=3, tide_amp=tide[0], tide_period=tide[1], tide_phase=tide[2])
    c = m.project_state(w["ic"])
    t0 = 500.0
    r_o = m.rhs(P, c, t=t0)
    out = {}
    for name, prec in (("fp32", swedg.PREC_MIXED_FP32), ("tf32", swedg.PREC_MIXED_TF32)):
        s = solver(w, prec, tide)
        s.set_state(c, t0)
        out[name] = s.rhs(c)
        s.close()
    hi = np.zeros_like(r_o, bool)
    hi[:, 3:, :] = True
    for name, r in out.items():
        e_all = rel_l2(r, r_o)
        e_hi = float(np.linalg.norm((r - r_o)[hi]) / np.linalg.norm(r_o[hi]))
        print(name, "rhs rel L2", e_all, "higher rows", e_hi)
        assert e_all < 5e-6, (name, e_all)
        assert e_hi < 1e-5, (name, e_hi)
    # the base rows only see the tensor cores through the FP32 correction of the
    # base modes: within FP32 round-off of the FP32 mode's
    lo = ~hi
    assert np.abs(out["tf32"][lo] - out["fp32"][lo]).max() <= 1e-5 * np.abs(r_o[lo]).max()


def test_tc_steps_accuracy_and_mass():
    w = workload(24, 4, pmin=1, pmax=4, open_west=False)
    m = O.Mesh(w["xy"], w["tri"], w["hv"], w["orders"])
    P = O.Params(g=w["g"], cfl=w["cfl"], rk_order=3)
    s = solver(w, swedg.PREC_MIXED_TF32)
    c = m.project_state(w["ic"])
    s.set_state(c, 0.0)
    n = 200  # CFL steps (a fixed step that suits p = 3 is unstable for p = 4)
    s.run(n)
    c_g, _ = s.get_state()
    c_o, _ = m.run(P, c, 0.0, n)
    err = rel_l2(c_g, c_o)
    print("tf32 200 steps rel L2", err)
    assert err < 1e-6, err
    m0 = m.mass(c)
    assert abs(s.mass() - m0) <= 1e-13 * math.sqrt(n) * abs(m0)
    s.close()


def test_tc_cfl_run_and_graph_replay_match_step_by_step():
    """swe_run (CUDA graph) and single swe_rk_step calls give the same state"""
    w = workload(20, 5)
    m = O.Mesh(w["xy"], w["tri"], w["hv"], w["orders"], bc_tag=w["bc_tag"])
    c = m.project_state(w["ic"])
    a = solver(w, swedg.PREC_MIXED_TF32, tide=(0.2, 900.0, 0.0))
    b = solver(w, swedg.PREC_MIXED_TF32, tide=(0.2, 900.0, 0.0))
    a.set_state(c, 0.0)
    b.set_state(c, 0.0)
    a.run(12)
    for _ in range(12):
        b.rk_step()
    ca, ta = a.get_state()
    cb, tb = b.get_state()
    assert ta == tb
    assert np.array_equal(ca, cb)
    assert a.memory_bytes() == serve.device_bytes([w], swedg.PREC_MIXED_TF32)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [swedg.PREC_MIXED_FP32, swedg.PREC_MIXED_TF32])
def test_autotuned_shape_gives_the_same_state(prec):
    """the launch shape (schedule included) changes no result: every unit is
    computed by one thread in the same order"""
    w = workload(30, 6)
    m = O.Mesh(w["xy"], w["tri"], w["hv"], w["orders"], bc_tag=w["bc_tag"])
    c = m.project_state(w["ic"])
    a = solver(w, prec)
    b = solver(w, prec)
    a.set_state(c, 0.0)
    b.set_state(c, 0.0)
    c0, _ = a.get_state()
    shape, ms = a.autotune(steps=3)
    print("autotuned shape", shape, "ms per step", ms)
    assert a.launch_shape() == shape and ms > 0
    c_a, t_a = a.get_state()
    assert t_a == 0.0 and np.array_equal(c_a, c0)  # the trial steps left no trace
    b.set_launch_shape((1, 64, 128, 64, 1 - shape[4], 0 if shape[5] else 3))  # the other schedules
    a.run(10)
    b.run(10)
    assert np.array_equal(a.get_state()[0], b.get_state()[0])
    with pytest.raises(swedg.SweError):
        a.set_launch_shape((2, 100, 256, 128, 0, 2))
    with pytest.raises(swedg.SweError):
        a.set_launch_shape((2, 128, 256, 128, 2, 2))
    with pytest.raises(swedg.SweError):
        a.set_launch_shape((2, 128, 256, 128, 0, 17))
    with pytest.raises(ValueError):
        a.set_launch_shape((2, 128, 256, 128, 0))
    a.close()
    b.close()
