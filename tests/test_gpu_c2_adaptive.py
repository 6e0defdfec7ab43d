"""The p-adaptive ocean recipe (131,072 triangles in the benchmark) at 64x64
split squares (8,192 triangles) over a whole run: 1000 SSP-RK3 CFL steps with
the modal-decay indicator every 10 steps (orders p in {1, 2, 3}), in the FP64
mode and in the mixed mode (FP32 correction), against the FP64 oracle doing
the same run (paper Sect. 2 end and Sect. 5: dynamically p-adaptive runs).

FP64 mode: one swe_run_adaptive call; the order map after every pass is a
decision both sides take in FP64, so the final maps must be equal and the
state within 1e-11 relative L2.  No indicator value of the oracle's run comes
within 1e-9 of a threshold, so no decision is ambiguous at FP64 round-off.

Mixed mode: the correction modes are FP32, so an indicator value within the
mode's error of a threshold may be decided the other way, and both decisions
are then correct.  The run goes pass by pass (swe_run of 10 steps, swe_adapt);
every decision of the library must equal the oracle's, except where the
oracle's value lies within 1e-3 (relative) of the threshold; there the oracle
follows the library's choice.  The state must stay within 1e-6 relative L2.
"""
import numpy as np
import pytest

import oracle as O
from paper_2311_11348_gb300 import build, inputs, swedg

pytestmark = pytest.mark.gpu

UP, DOWN, PMIN, PMAX, EVERY, PASSES = 0.05, 1e-3, 1, 3, 10, 100


@pytest.fixture(scope="module")
def setup():
    build.build()
    swedg.load()
    w = inputs.ocean_p123(64)
    m = O.Mesh(w["xy"], w["tri"], w["hv"], w["orders"], threads=0)
    c0 = m.project_state(w["ic"], n=8)
    return w, c0


def solver(w, precision):
    s = swedg.Solver(g=w["g"], cfl=w["cfl"], rk_order=3, precision=precision)
    s.set_mesh(w["xy"], w["tri"])
    s.set_bathymetry(w["hv"])
    s.set_orders(w["orders"])
    return s


def margin(sv, orders):
    """relative distance of the indicator values of p >= 2 elements (p = 1
    elements always give 1) from the nearer threshold"""
    mg = np.minimum(np.abs(sv - UP) / UP, np.abs(sv - DOWN) / DOWN)
    return mg[orders > 1]


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_adaptive_run_fp64_matches_the_oracle(setup):
    w, c0 = setup
    m = O.Mesh(w["xy"], w["tri"], w["hv"], w["orders"], threads=0)
    P = O.Params(g=w["g"], cfl=w["cfl"], rk_order=3)
    c, t, changed = c0.copy(), 0.0, []
    for _ in range(PASSES):
        c, t = m.run(P, c, t, EVERY)
        new, sv, n = m.indicator(c, UP, DOWN, PMIN, PMAX)
        assert margin(sv, m.orders).min() > 1e-9
        c = m.adapt_state(c, new)
        changed.append(n)
    assert min(changed) > 0 and len(set(new)) == 3
    s = solver(w, swedg.PREC_FP64)
    s.set_state(c0, 0.0)
    t_g = s.run_adaptive(EVERY * PASSES, EVERY, UP, DOWN, PMIN, PMAX)
    got, _ = s.get_state()
    o_g, n0 = s.adapt(1e300, -1.0, PMIN, PMAX)  # thresholds that change nothing: the current map
    s.close()
    assert n0 == 0
    assert np.array_equal(o_g, new)
    assert abs(t_g - t) <= 1e-11 * t
    err = rel_l2(got, c)
    print(f"FP64 adaptive run: rel L2 {err:.2e}, orders {np.bincount(new, minlength=4)[1:]}, t {t:.3f} s")
    assert err < 1e-11


def test_adaptive_run_mixed_matches_the_oracle(setup):
    w, c0 = setup
    m = O.Mesh(w["xy"], w["tri"], w["hv"], w["orders"], threads=0)
    P = O.Params(g=w["g"], cfl=w["cfl"], rk_order=3)
    s = solver(w, swedg.PREC_MIXED_FP32)
    s.set_state(c0, 0.0)
    c, t = c0.copy(), 0.0
    adopted = decisions = 0
    for _ in range(PASSES):
        c, t = m.run(P, c, t, EVERY)
        s.run(EVERY)
        o_g, _ = s.adapt(UP, DOWN, PMIN, PMAX)
        o_o, sv, _ = m.indicator(c, UP, DOWN, PMIN, PMAX)
        diff = np.nonzero(o_g != o_o)[0]
        decisions += int((m.orders > 1).sum())
        if len(diff):
            # both choices are valid only for a value at the threshold within the mode's error
            mg = np.minimum(np.abs(sv[diff] - UP) / UP, np.abs(sv[diff] - DOWN) / DOWN)
            assert mg.max() <= 1e-3, (diff, sv[diff])
            adopted += len(diff)
        c = m.adapt_state(c, o_g)
    got, t_g = s.get_state()
    s.close()
    err = rel_l2(got, c)
    print(f"mixed adaptive run: rel L2 {err:.2e}, {adopted} of {decisions} decisions at a threshold, t {t:.3f} s")
    assert adopted <= 1e-4 * decisions
    assert abs(t_g - t) <= 1e-6 * t
    assert err < 1e-6
