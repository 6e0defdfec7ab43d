"""Serving loop: continuous batching of shallow water simulations on one GPU.

Requests (a mesh, an initial state and a step count) arrive over time.  The
server admits waiting requests while the device footprint stays within the
memory budget; the requests admitted at one scheduling point form a cohort,
one union context (ensemble.Ensemble / swe_set_members) in which the RK
stages of all its requests run in shared launches, each request with its own
CFL step and time.  All cohorts advance together, chunk by chunk, each from
its own host thread on its own CUDA streams, so their launches overlap on the
GPU.  A finished request's state is copied out at once; its cohort is
compacted (rebuilt with the continuing requests, states moved device to
device) when requests wait for memory or less than half of it is still live,
and the two smallest cohorts are merged when there are more than max_cohorts.
Every context build runs on the host thread pool while the other cohorts
take their next chunk: a new cohort joins at the end of the round that
admitted it, a compacted or merged one (whose requests pause meanwhile) at
the end of the following round.  So admitting a request costs one context
build of its own cohort, not of everything on the GPU, and no build holds up
the cohorts already running.

This module is host-side scheduling only; every step runs in the CUDA library.
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import threading
import time

import numpy as np

from . import swedg
from .ensemble import Ensemble

KMAX = swedg.KMAX
KP = (1, 3, 6, 10, 15)
NGEO, NEGEO = 20, 11  # rows of the element and edge geometry tables


def device_bytes(meshes, precision):
    """Device bytes a context holds after swe_set_mesh + swe_set_orders (+
    swe_set_members) of the disjoint union of `meshes`: the same allocations
    the library makes (swe_memory_bytes reports them), counted on the host so
    that admission needs no context.  Per element: the mesh in caller order
    and regrouped (geometry and its FP32 copy, topology), three RK states,
    velocity, the user-layout staging; per edge: geometry and base fluxes;
    per element of order p >= 2 also the projections of its three edges'
    fluxes onto its higher modes.  The correction arrays scale with K - 3 at
    the correction type's width (4 bytes in the mixed mode, 8 in FP64).  After an order change the library may hold
    more (its order-group buffers grow with a quarter to spare)."""
    corr32 = precision in (swedg.PREC_MIXED_FP32, swedg.PREC_MIXED_TF32)
    ts = 4 if corr32 else 8
    ne = nE = 0
    n = [0] * 5
    for m in meshes:
        tri = np.asarray(m["tri"], np.int64)
        p = np.asarray(m["orders"], np.int64)
        ne += len(tri)
        for q in range(5):
            n[q] += int((p == q).sum())
        a = tri.reshape(-1)
        b = tri[:, [1, 2, 0]].reshape(-1)
        key = np.minimum(a, b) * (int(tri.max(initial=0)) + 1) + np.maximum(a, b)
        key = np.sort(key)
        first = np.ones(len(key), bool)
        first[1:] = key[1:] != key[:-1]
        nE += int(first.sum())
    nm = max(len(meshes), 1)
    nrc = n[2] + n[3] + n[4]
    be, bg = -(-ne // 256), -(-nE // 256)
    allocs = [NGEO * 8 * ne, 96 * ne, 12 * ne, 4 * nE, 4 * nE, 4 * ne,                    # mesh in caller order
              4 * nE, NEGEO * 8 * nE, NEGEO * 4 * nE, 4 * nE,                                # edge info, geometry, members
              4 * ne, 4 * ne, ne, NGEO * 8 * ne, NGEO * 4 * ne, 96 * ne, 4 * ne, 12 * ne,    # regrouped elements
              4 * nE, 4 * nE, 4 * nE, 12 * nE, 8 * ne,                                       # regrouped edges, offsets
              20 * be, 40 * be, 12 * bg, 24 * bg, 8 * be, 8 * (be + 1), 128]                # partition scratch
    allocs += [72 * ne] * 3 + ([36 * ne] * 3 if corr32 else [])                             # base RK states
    allocs += [48 * ne] + ([24 * ne] if corr32 else [])                                     # base velocity
    allocs += [48 * nE, 48 * nE, 8 * 3 * KMAX * ne, 8 * 3 * KMAX * ne, ne,                  # fluxes, staging, orders
               8 * nm, 8 * nm, 8 * nm, 4, 4 * nm,                                           # members, status words
               8 * min(1024, max(1, (ne + 255) // 256)), 16, 16]                           # sums, tickets
    for q in (2, 3, 4):                                                                     # order groups
        allocs += [ts * 3 * (KP[q] - 3) * n[q]] * 3
        allocs += [ts * 2 * (KP[q] - 3) * n[q], ts * 4 * KP[q] * n[q], ts * KP[q] * n[q]]
        allocs += [ts * 3 * 3 * (KP[q] - 3) * n[q]]                                        # projected edge fluxes
    allocs += [32 * max(nrc, 1)]
    if precision == swedg.PREC_MIXED_TF32:
        allocs += [32 * 4 * max(nrc, 1)]                                                    # tensor-core volume terms
    b = sum(a if a > 0 else 16 for a in allocs)  # the library allocates 16 bytes for an empty array
    return b


@dataclasses.dataclass
class Request:
    rid: int
    mesh: dict          # xy, tri, hv, orders (and bc_tag)
    state: np.ndarray   # c[3][15][ne] initial state
    steps: int
    arrival: float = 0.0
    # filled by the server
    admitted: float = -1.0
    finished: float = -1.0
    result: np.ndarray = None
    t_final: float = 0.0
    done_steps: int = 0
    nbytes: int = None
    error: str = None   # set when the request was evicted after a failed step


def footprint(req: Request, precision: int) -> int:
    """device bytes the request adds to a union context (computed once)"""
    if req.nbytes is None:
        req.nbytes = device_bytes([req.mesh], precision)
    return req.nbytes


class Cohort:
    """one union context over some requests; `live` marks those still running"""

    def __init__(self, reqs, kw, precision, device_resident, keep):
        self.reqs = list(reqs)
        self.live = [True] * len(self.reqs)
        self.nbytes = sum(footprint(r, precision) for r in self.reqs)
        self.ens = Ensemble([r.mesh for r in self.reqs], **kw)
        states = [keep.get(r.rid, r.state) for r in self.reqs]
        if device_resident:
            import torch
            states = [x if hasattr(x, "is_cuda") else torch.from_numpy(np.ascontiguousarray(x)).cuda()
                      for x in states]
        self.ens.set_states(states, [keep.get(("t", r.rid), 0.0) for r in self.reqs])

    def live_fraction(self):
        ne = [len(r.mesh["tri"]) for r in self.reqs]
        return sum(n for n, l in zip(ne, self.live) if l) / max(sum(ne), 1)


class Server:
    def __init__(self, budget_bytes: int, precision=swedg.PREC_MIXED_FP32, g=9.81, cfl=0.1, rk_order=3,
                 max_chunk=50, clock=time.perf_counter, device_resident=True, max_cohorts=8, h_min=1e-8):
        self.budget = budget_bytes
        self.device_resident = device_resident
        self.kw = dict(g=g, cfl=cfl, rk_order=rk_order, precision=precision, h_min=h_min)
        self.precision = precision
        self.max_chunk = max_chunk
        self.max_cohorts = max_cohorts
        self.clock = clock
        self.waiting: list[Request] = []
        self.cohorts: list[Cohort] = []
        self.pending: list = []  # [future of a Cohort, its bytes, the round it joins at the end of, its requests]
        self.done: list[Request] = []
        self.failed: list[Request] = []
        self.h_min = h_min
        self.dof_stage_updates = 0
        self.rebuilds = 0
        self.rebuild_s = 0.0    # host time spent building cohort contexts (mostly beside the GPU work)
        self.launches = 0       # kernels launched by closed cohort contexts
        self.round = 0
        self._lock = threading.Lock()
        self.pool = concurrent.futures.ThreadPoolExecutor(max_workers=max_cohorts + 4)

    @property
    def active(self):
        return [r for c in self.cohorts for r, l in zip(c.reqs, c.live) if l]

    @property
    def in_flight(self):
        """admitted and unfinished: running, or in a cohort being built"""
        return self.active + [r for p in self.pending for r in p[3]]

    def submit(self, req: Request):
        req.arrival = self.clock() if req.arrival <= 0.0 else req.arrival
        self.waiting.append(req)

    def _used(self):
        return sum(c.nbytes for c in self.cohorts) + sum(p[1] for p in self.pending)

    def _close(self, c):
        prof = getattr(c.ens.solver, "profile_read", None) if hasattr(c.ens, "solver") else None
        if prof is not None:
            self.launches += int(prof()["kernels"][1])
        c.ens.close()

    def _build(self, reqs, keep):
        t0 = self.clock()
        c = Cohort(reqs, self.kw, self.precision, self.device_resident, keep)
        with self._lock:
            self.rebuilds += 1
            self.rebuild_s += self.clock() - t0
        return c

    def _build_later(self, reqs, keep, due):
        nbytes = sum(footprint(r, self.precision) for r in reqs)
        self.pending.append([self.pool.submit(self._build, reqs, keep), nbytes, due, list(reqs)])

    def _rebuild_later(self, cohorts, due):
        """the live requests of `cohorts` into one new cohort, built on the pool
        (states and times taken now, on the device); the old contexts close"""
        keep, reqs = {}, []
        for c in cohorts:
            states = c.ens.states(device=self.device_resident)
            t, _ = c.ens.times()
            for i, r in enumerate(c.reqs):
                if c.live[i]:
                    keep[r.rid] = states[i]
                    keep[("t", r.rid)] = t[i]
                    reqs.append(r)
            self._close(c)
        if reqs:
            self._build_later(reqs, keep, due)

    def _join(self, upto=None):
        """cohorts whose build is due by round `upto` (all when None) join the running ones"""
        keep = []
        for p in self.pending:
            if upto is None or p[2] <= upto:
                self.cohorts.append(p[0].result())
            else:
                keep.append(p)
        self.pending = keep

    @staticmethod
    def _run_cohort(c, chunk):
        try:
            c.ens.run(chunk)
            return None
        except swedg.SweError as err:
            return err

    def _evict_failed(self, c, err):
        """A cohort's run reported an error (a non-finite state or a depth at or
        below h_min in some member).  The members evolve independently, so
        the ones the library's per-member status words do not flag keep the
        chunk they just ran; the flagged ones are evicted with the error,
        without touching other requests.  Without a member to blame (a device
        wait that timed out), the whole cohort is evicted."""
        status = c.ens.member_status()
        bad = [i for i in range(len(c.reqs)) if c.live[i] and status[i] != 0]
        if not bad:
            bad = [i for i in range(len(c.reqs)) if c.live[i]]
        now = self.clock()
        for i in bad:
            r = c.reqs[i]
            c.live[i] = False
            r.error = f"{err}"
            r.finished = now
            self.failed.append(r)

    def step(self):
        """One scheduling round: admit, run a chunk on every cohort, retire.  Returns False when idle."""
        rnd = self.round
        self.round += 1
        admitted = []
        used = self._used()
        while self.waiting:
            r = self.waiting[0]
            f = footprint(r, self.precision)
            if (self.cohorts or self.pending or admitted) and used + f > self.budget:
                break
            self.waiting.pop(0)
            r.admitted = self.clock()
            admitted.append(r)
            used += f
        if admitted:
            if self.cohorts:  # built on the host while the running cohorts take their chunk
                self._build_later(admitted, {}, rnd)
            else:
                self.cohorts.append(self._build(admitted, {}))
        active = self.active
        if not active:
            self._join()
            return bool(self.cohorts or self.waiting)
        chunk = min(self.max_chunk, min(r.steps - r.done_steps for r in active))
        errors = list(self.pool.map(lambda c: self._run_cohort(c, chunk), self.cohorts))
        failed = set()
        for c, err in zip(self.cohorts, errors):
            if err is not None:
                self._evict_failed(c, err)
                failed.add(id(c))
        active = self.active
        for r in active:
            r.done_steps += chunk
            K = np.array(KP)[np.asarray(r.mesh["orders"], np.int64)]
            self.dof_stage_updates += chunk * self.kw["rk_order"] * 3 * int(K.sum())
        # retire; compactions are built on the pool and join at the end of the next round
        now = None
        keep_cohorts = []
        for c in self.cohorts:
            fin = [i for i, r in enumerate(c.reqs) if c.live[i] and r.done_steps >= r.steps]
            if fin:
                states = c.ens.states(device=self.device_resident)
                t, _ = c.ens.times()
                now = self.clock()
                for i in fin:
                    r = c.reqs[i]
                    r.result = states[i].cpu().numpy() if hasattr(states[i], "cpu") else states[i]
                    r.t_final = float(t[i])
                    r.finished = now
                    c.live[i] = False
                    self.done.append(r)
            if not any(c.live):
                self._close(c)
            elif id(c) in failed or (fin and (self.waiting or c.live_fraction() < 0.5)):  # evicted: always compact
                self._rebuild_later([c], rnd + 1)
            else:
                keep_cohorts.append(c)
        self.cohorts = keep_cohorts
        self._join(upto=rnd)
        while len(self.cohorts) + len(self.pending) > self.max_cohorts and len(self.cohorts) >= 2:
            a, b = sorted(self.cohorts, key=lambda c: c.nbytes)[:2]
            self.cohorts = [c for c in self.cohorts if c is not a and c is not b]
            self._rebuild_later([a, b], rnd + 1)
        return True

    def run_until_idle(self):
        while self.step():
            pass

    def latencies(self):
        return np.array([r.finished - r.arrival for r in self.done])

    def close(self):
        self._join()
        for c in self.cohorts:
            self._close(c)
        self.cohorts = []
        self.pool.shutdown(wait=True)
