"""Scheduling logic of the serving loop on the CPU (no GPU): admission by
device footprint, chunking by the smallest remaining step count, retirement
and re-batching.  The union context is replaced by a recording fake."""
import numpy as np

from paper_2311_11348_gb300 import serve, swedg


class FakeUnion:
    log = []

    def __init__(self, meshes, **kw):
        self.meshes = meshes
        self.ne = [len(m["tri"]) for m in meshes]
        self.t = np.zeros(len(meshes))
        FakeUnion.log.append(("build", len(meshes)))

    def set_states(self, states, times=None):
        self.c = [np.array(s, copy=True) for s in states]
        self.t = np.zeros(len(states)) if times is None else np.array(times, float)

    def states(self, device=False):
        return [c.copy() for c in self.c]

    def times(self):
        return self.t.copy(), np.ones_like(self.t)

    def run(self, n, dt_fixed=0.0):
        FakeUnion.log.append(("run", n, len(self.c)))
        for c in self.c:
            c += n  # a state that counts steps
        self.t += n

    def close(self):
        pass


def make_req(rid, ne, steps):
    mesh = dict(xy=np.zeros((3, 2)), tri=np.zeros((ne, 3), np.int32), hv=np.ones(3), orders=np.ones(ne, np.int8))
    return serve.Request(rid=rid, mesh=mesh, state=np.zeros((3, 15, ne)), steps=steps, arrival=1.0)


def test_admission_chunking_and_results(monkeypatch):
    monkeypatch.setattr(serve, "Ensemble", FakeUnion)
    FakeUnion.log = []
    reqs = [make_req(rid, ne, steps) for rid, ne, steps in [(0, 100, 30), (1, 100, 70), (2, 120, 20)]]
    f = [serve.footprint(r, swedg.PREC_MIXED_FP32) for r in reqs]
    assert f[0] < f[2]
    srv = serve.Server(budget_bytes=f[1] + f[2], precision=swedg.PREC_MIXED_FP32, max_chunk=40, clock=lambda: 2.0,
                       device_resident=False)
    for r in reqs:
        srv.submit(r)
    srv.run_until_idle()
    srv.close()
    done = {r.rid: r for r in srv.done}
    assert set(done) == {0, 1, 2}
    for r in done.values():
        assert np.all(r.result == r.steps) and r.t_final == r.steps  # every request ran exactly its steps
    runs = [e for e in FakeUnion.log if e[0] == "run"]
    builds = [e for e in FakeUnion.log if e[0] == "build"]
    # 0 and 1 fit the budget together and form one cohort; the chunk stops at 0's end;
    # 1's cohort is compacted because 2 waits, built on the pool during the next
    # round, in which 2's cohort (built at once: nothing else runs) takes its 20
    # steps; 1 rejoins at the end of that round and runs to its end
    assert runs[0] == ("run", 30, 2)
    assert runs[1:] == [("run", 20, 1), ("run", 40, 1)]
    assert builds == [("build", 2), ("build", 1), ("build", 1)]
    assert srv.latencies().shape == (3,)


def test_cohorts_merge_beyond_the_limit(monkeypatch):
    monkeypatch.setattr(serve, "Ensemble", FakeUnion)
    FakeUnion.log = []
    srv = serve.Server(budget_bytes=1 << 40, max_chunk=10, clock=lambda: 0.0, device_resident=False, max_cohorts=2)
    for k in range(4):  # one arrival per scheduling round: four cohorts, merged down to two
        srv.submit(make_req(k, 50 + k, 100))
        srv.step()
        assert len(srv.cohorts) <= 2
    srv.run_until_idle()
    srv.close()
    assert sorted(r.rid for r in srv.done) == [0, 1, 2, 3]
    for r in srv.done:
        assert np.all(r.result == r.steps) and r.t_final == r.steps


def test_a_request_larger_than_the_budget_still_runs_alone(monkeypatch):
    monkeypatch.setattr(serve, "Ensemble", FakeUnion)
    FakeUnion.log = []
    srv = serve.Server(budget_bytes=10, max_chunk=50, clock=lambda: 0.0, device_resident=False)
    srv.submit(make_req(0, 1000, 10))
    srv.submit(make_req(1, 1000, 10))
    srv.run_until_idle()
    runs = [e for e in FakeUnion.log if e[0] == "run"]
    assert runs == [("run", 10, 1), ("run", 10, 1)]


def test_device_bytes_counts_edges_orders_and_precision():
    from paper_2311_11348_gb300 import inputs
    xy, tri = inputs.split_square_mesh(4, 1.0)
    p1 = dict(tri=tri, orders=np.ones(len(tri), np.int8))
    p3 = dict(tri=tri, orders=np.full(len(tri), 3, np.int8))
    b64 = serve.device_bytes([p1], swedg.PREC_FP64)
    assert serve.device_bytes([p1], swedg.PREC_MIXED_FP32) > b64  # FP32 copies of the P1 data
    assert serve.device_bytes([p3], swedg.PREC_FP64) > serve.device_bytes([p3], swedg.PREC_MIXED_FP32) > b64
    # a union holds the same per-element and per-edge arrays as its members;
    # only the fixed per-context arrays (and 16-byte empty ones) are shared
    both = serve.device_bytes([p1, p3], swedg.PREC_FP64)
    alone = b64 + serve.device_bytes([p3], swedg.PREC_FP64)
    assert 0 < alone - both < 1024
    assert serve.device_bytes([p3], swedg.PREC_MIXED_TF32) > serve.device_bytes([p3], swedg.PREC_MIXED_FP32)


class PoisonUnion(FakeUnion):
    """a fake whose run fails when a member's mesh is marked poisoned: that
    member's state turns non-finite, the others advance as usual"""

    def run(self, n, dt_fixed=0.0):
        super().run(n, dt_fixed)
        bad = [i for i, m in enumerate(self.meshes) if m.get("poison")]
        self.status = np.zeros(len(self.meshes), np.uint32)
        for i in bad:
            self.c[i][:] = np.nan
            self.status[i] = swedg.STATUS_NONFINITE
        if bad:
            raise swedg.SweError(-4, "non-finite value in the state")

    def member_status(self):
        return self.status


def test_a_failing_request_is_evicted_without_the_others(monkeypatch):
    monkeypatch.setattr(serve, "Ensemble", PoisonUnion)
    FakeUnion.log = []
    srv = serve.Server(budget_bytes=1 << 40, max_chunk=25, clock=lambda: 0.0, device_resident=False)
    reqs = []
    for rid in range(3):
        r = make_req(rid, 20, 60)
        # a valid mesh for the depth check: vertices far apart, deep water
        r.mesh["xy"] = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
        r.mesh["hv"] = np.full(3, 10.0)
        r.mesh["tri"] = np.tile(np.array([[0, 1, 2]], np.int32), (20, 1))
        reqs.append(r)
    reqs[1].mesh["poison"] = True
    for r in reqs:
        srv.submit(r)
    srv.run_until_idle()
    srv.close()
    assert [r.rid for r in srv.failed] == [1] and "non-finite" in srv.failed[0].error
    done = {r.rid: r for r in srv.done}
    assert set(done) == {0, 2}
    for r in done.values():
        assert np.all(r.result == r.steps) and r.t_final == r.steps
