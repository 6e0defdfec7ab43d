"""Batched ensembles and the serving loop on the GPU: every member's result
is the same alone and in the mix (bitwise: the per-element arithmetic and the
per-member CFL minimum do not depend on the other members), and every
member's and every served request's result matches the FP64 oracle run of
that simulation alone (relative L2: 1e-11 in the FP64 mode, 1e-6 in the
mixed and tensor-core modes; the final time to the same bounds)."""
import numpy as np
import pytest

import oracle as O
from paper_2311_11348_gb300 import build, ensemble, inputs, serve, swedg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    swedg.load()


def member(n, L, seed, pmin, pmax, open_west=False):
    xy, tri = inputs.split_square_mesh(n, L, jitter=0.2, seed=seed)
    hv = inputs.fourier_bathymetry(xy, L, lo=30.0, hi=300.0, seed=seed + 1)
    rng = np.random.default_rng(seed)
    orders = rng.integers(pmin, pmax + 1, size=len(tri)).astype(np.int8)
    bc = inputs.boundary_tags(xy, tri, "west") if open_west else None
    m = O.Mesh(xy, tri, hv, orders, bc_tag=bc)
    c = m.project_state(lambda x, y: (0.4 * np.exp(-((x - 0.6 * L) ** 2 + (y - 0.4 * L) ** 2) / (0.02 * L * L)),
                                      0.0 * x + 2.0, 0.0 * y - 1.0), n=5)
    return dict(xy=xy, tri=tri, hv=hv, orders=orders, bc_tag=bc), c


TOL = {swedg.PREC_FP64: 1e-11, swedg.PREC_MIXED_FP32: 1e-6, swedg.PREC_MIXED_TF32: 1e-6}


def oracle_run(mesh, c, steps, g=9.81, cfl=0.2, rk_order=3, tide=(0.0, 0.0, 0.0), **_):
    """the same simulation in the FP64 oracle: steps CFL steps from t = 0"""
    m = O.Mesh(mesh["xy"], mesh["tri"], mesh["hv"], mesh["orders"], bc_tag=mesh.get("bc_tag"))
    P = O.Params(g=g, cfl=cfl, rk_order=rk_order, tide_amp=tide[0], tide_period=tide[1], tide_phase=tide[2])
    return m.run(P, c, 0.0, steps)


def check_against_oracle(got, t_got, mesh, c, steps, precision, **kw):
    ref, t_ref = oracle_run(mesh, c, steps, **kw)
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert err < TOL[precision], (precision, err)
    assert abs(t_got - t_ref) <= TOL[precision] * t_ref, (precision, t_got, t_ref)
    return err


def alone(mesh, c, steps, **kw):
    s = swedg.Solver(**kw)
    s.set_mesh(mesh["xy"], mesh["tri"], mesh.get("bc_tag"))
    s.set_bathymetry(mesh["hv"])
    s.set_orders(mesh["orders"])
    s.set_state(c, 0.0)
    t = s.run(steps)
    out, _ = s.get_state()
    nbytes = s.memory_bytes()
    s.close()
    return out, t, nbytes


@pytest.mark.parametrize("precision", [swedg.PREC_FP64, swedg.PREC_MIXED_FP32, swedg.PREC_MIXED_TF32])
def test_ensemble_member_equals_alone(precision):
    """(in the tensor-core mode the union puts other members' elements into the same 128-element MMA
    tiles; every output row of an MMA depends only on its own row of A)"""
    kw = dict(g=9.81, cfl=0.2, rk_order=3, precision=precision, tide=(0.2, 900.0, 0.0))
    specs = [member(8, 2e3, 1, 1, 2), member(14, 5e3, 2, 1, 3, open_west=True), member(5, 1e3, 3, 2, 4)]
    ens = ensemble.Ensemble([m for m, _ in specs], **kw)
    ens.set_states([c for _, c in specs])
    ens.run(15)
    got = ens.states()
    t_ens, dt_ens = ens.times()
    assert ens.solver.memory_bytes() == serve.device_bytes([m for m, _ in specs], precision)
    ens.close()
    assert len(set(np.round(dt_ens, 12))) == 3  # every member took its own CFL step
    for i, (m, c) in enumerate(specs):
        ref, t, nbytes = alone(m, c, 15, **kw)
        assert t_ens[i] == t
        assert np.array_equal(got[i], ref)
        assert nbytes == serve.device_bytes([m], precision)
        check_against_oracle(got[i], t_ens[i], m, c, 15, **kw)


def test_serving_results_equal_alone_with_admission_by_footprint():
    kw = dict(g=9.81, cfl=0.2, rk_order=3, precision=swedg.PREC_MIXED_FP32)
    specs = [member(8, 2e3, 11, 1, 2), member(10, 3e3, 12, 1, 3), member(6, 1e3, 13, 1, 2), member(9, 2e3, 14, 2, 3)]
    steps = [25, 10, 40, 15]
    fp = [serve.device_bytes([m], kw["precision"]) for m, _ in specs]
    budget = fp[0] + fp[1] + 1  # two at a time
    srv = serve.Server(budget, precision=kw["precision"], g=9.81, cfl=0.2, rk_order=3, max_chunk=8)
    for i, ((m, c), st) in enumerate(zip(specs, steps)):
        srv.submit(serve.Request(rid=i, mesh=m, state=c, steps=st))
        if i == 1:
            srv.step()  # the later requests arrive while the first two run
    srv.run_until_idle()
    srv.close()
    assert srv.rebuilds >= 3
    done = {r.rid: r for r in srv.done}
    for i, ((m, c), st) in enumerate(zip(specs, steps)):
        ref, t, _ = alone(m, c, st, **kw)
        assert done[i].t_final == t
        assert np.array_equal(done[i].result, ref)
        check_against_oracle(done[i].result, done[i].t_final, m, c, st, **kw)
    lat = srv.latencies()
    assert np.all(lat > 0)


def test_serving_evicts_a_failing_request_and_finishes_the_others():
    """One request starts with a negative depth (xi = -500 m on a 30..300 m
    sea): its cohort's run reports the error, the server evicts that request
    and the others finish exactly as alone."""
    kw = dict(g=9.81, cfl=0.2, rk_order=3, precision=swedg.PREC_MIXED_FP32)
    specs = [member(8, 2e3, 21, 1, 2), member(6, 1e3, 22, 1, 3), member(7, 2e3, 23, 1, 2)]
    bad_mesh, bad_c = specs[1]
    bad_c = bad_c.copy()
    bad_c[0, 0] = -500.0 * np.sqrt(0.5 * (1e3 / 6) ** 2)  # mean elevation -500 m everywhere
    srv = serve.Server(1 << 40, precision=kw["precision"], g=9.81, cfl=0.2, rk_order=3, max_chunk=10)
    for i, (m, c) in enumerate(specs):
        srv.submit(serve.Request(rid=i, mesh=m, state=bad_c if i == 1 else c, steps=20))
    srv.run_until_idle()
    srv.close()
    assert [r.rid for r in srv.failed] == [1]
    assert srv.failed[0].error
    done = {r.rid: r for r in srv.done}
    assert set(done) == {0, 2}
    for i in (0, 2):
        m, c = specs[i]
        ref, t, _ = alone(m, c, 20, **kw)
        assert done[i].t_final == t
        assert np.array_equal(done[i].result, ref)
        check_against_oracle(done[i].result, done[i].t_final, m, c, 20, **kw)


def test_member_status_names_the_failing_member():
    """swe_member_status: after a run that reports a depth failure, only the
    member whose state went below h_min carries the status bit; reading clears
    the bits, and a new state upload starts them afresh"""
    kw = dict(g=9.81, cfl=0.2, rk_order=3, precision=swedg.PREC_MIXED_FP32)
    specs = [member(6, 1e3, 31, 1, 2), member(7, 2e3, 32, 1, 3), member(5, 1e3, 33, 1, 2)]
    ens = ensemble.Ensemble([m for m, _ in specs], **kw)
    states = [c.copy() for _, c in specs]
    states[1][0, 0] = -500.0 * np.sqrt(0.5 * (2e3 / 7) ** 2)  # mean elevation -500 m on a 30..300 m sea
    ens.set_states(states)
    with pytest.raises(swedg.SweError) as ei:
        ens.run(2)
    assert ei.value.code in (-3, -4)  # the negative depth also turns the state non-finite
    st = ens.member_status()
    assert st[1] & swedg.STATUS_DEPTH and st[0] == 0 and st[2] == 0
    assert not np.any(ens.member_status())  # read and cleared
    ens.set_states([c for _, c in specs])
    ens.run(2)
    assert not np.any(ens.member_status())
    ens.close()
