"""Serving loop: continuous batching of shallow water simulations on one GPU.

Requests (a mesh, an initial state and a step count) arrive over time.  The
server keeps every admitted request's state on the device inside one union
context (ensemble.Ensemble / swe_set_members), so the RK stages of all active
requests run in shared launches, each request with its own CFL step and time.
Between chunks of steps it retires finished requests (their state is copied
out) and admits waiting ones while the device footprint stays within the
memory budget; the union context is rebuilt on every membership change and
the continuing requests' states are moved device to device.

This module is host-side scheduling only; every step runs in the CUDA library.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import swedg
from .ensemble import Ensemble

KMAX = swedg.KMAX
KP = (1, 3, 6, 10, 15)
NGEO, NEGEO = 19, 9  # rows of the element and edge geometry tables


def _npts(pm):
    return 2 if pm <= 1 else (3 * pm + 2) // 2


def device_bytes(meshes, precision):
    """Device bytes a context holds after swe_set_mesh + swe_set_orders (+
    swe_set_members) of the disjoint union of `meshes`: the same allocations
    the library makes (swe_memory_bytes reports them), counted on the host so
    that admission needs no context.  Per element: FP64 geometry and its FP32
    copy, topology, three RK states, velocity, the user-layout staging; per
    edge: geometry, base fluxes and the correction flux buffers of its max
    order; the correction arrays scale with K(p) - 3 at the correction type's
    width (4 bytes in the mixed mode, 8 in FP64)."""
    corr32 = precision == swedg.PREC_MIXED_FP32
    ts = 4 if corr32 else 8
    ne = nE = 0
    n = [0] * 5
    ncl = [0] * 5
    for m in meshes:
        tri = np.asarray(m["tri"], np.int64)
        p = np.asarray(m["orders"], np.int64)
        ne += len(tri)
        for q in range(5):
            n[q] += int((p == q).sum())
        a = tri.reshape(-1)
        b = tri[:, [1, 2, 0]].reshape(-1)
        key = np.minimum(a, b) * (int(tri.max(initial=0)) + 1) + np.maximum(a, b)
        owner = np.repeat(np.arange(len(tri)), 3)
        order = np.argsort(key, kind="stable")
        key, owner = key[order], owner[order]
        first = np.ones(len(key), bool)
        first[1:] = key[1:] != key[:-1]
        pm = np.maximum.reduceat(p[owner], np.flatnonzero(first)) if len(key) else np.zeros(0, np.int64)
        nE += int(first.sum())
        for q in (2, 3, 4):
            ncl[q] += int((pm == q).sum())
    nm = max(len(meshes), 1)
    nrc = n[2] + n[3] + n[4]
    b = NGEO * 12 * ne                      # geo + geo32
    b += ne * (1 + 12 + 4 + 4 + 1)          # p, eedge, perm, member, new orders
    b += nE * (12 + 4 + 4 + NEGEO * 12)     # eL/eR/einfo, slot, edge member, egeo + egeo32
    b += 12 * max(nrc, 1) + 4 * sum(ncl)    # element correction-edge slots, correction edge lists
    b += 3 * ne * (72 + (36 if corr32 else 0)) + sum(3 * ts * 3 * (KP[q] - 3) * n[q] for q in (2, 3, 4))
    b += ne * (48 + (24 if corr32 else 0)) + sum(ts * 2 * (KP[q] - 3) * n[q] for q in (2, 3, 4))
    b += 96 * nE + sum(ts * 3 * _npts(q) * ncl[q] for q in (2, 3, 4))
    b += 32 * max(nrc, 1) + 2 * 8 * 3 * KMAX * ne
    b += 24 * nm + 4 + 8 * min(1024, max(1, (ne + 255) // 256)) + 16
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


def footprint(req: Request, precision: int) -> int:
    """device bytes the request adds to a union context (computed once)"""
    if req.nbytes is None:
        req.nbytes = device_bytes([req.mesh], precision)
    return req.nbytes


class Server:
    def __init__(self, budget_bytes: int, precision=swedg.PREC_MIXED_FP32, g=9.81, cfl=0.1, rk_order=3,
                 max_chunk=50, clock=time.perf_counter, device_resident=True):
        self.budget = budget_bytes
        self.device_resident = device_resident
        self.kw = dict(g=g, cfl=cfl, rk_order=rk_order, precision=precision)
        self.precision = precision
        self.max_chunk = max_chunk
        self.clock = clock
        self.waiting: list[Request] = []
        self.active: list[Request] = []
        self.done: list[Request] = []
        self.union: Ensemble | None = None
        self.dof_stage_updates = 0
        self.rebuilds = 0

    def submit(self, req: Request):
        req.arrival = self.clock() if req.arrival <= 0.0 else req.arrival
        self.waiting.append(req)

    def _used(self):
        return sum(footprint(r, self.precision) for r in self.active)

    def _rebuild(self, keep_states):
        if self.union is not None:
            self.union.close()
            self.union = None
        if not self.active:
            return
        self.union = Ensemble([r.mesh for r in self.active], **self.kw)
        states = [keep_states.get(r.rid, r.state) for r in self.active]
        if self.device_resident:
            import torch
            states = [s if hasattr(s, "is_cuda") else torch.from_numpy(np.ascontiguousarray(s)).cuda() for s in states]
        times = [keep_states.get(("t", r.rid), 0.0) for r in self.active]
        self.union.set_states(states, times)
        self.rebuilds += 1

    def step(self):
        """One scheduling round: admit, run a chunk, retire.  Returns False when idle."""
        # admit while the device footprint fits the budget (at least one request)
        admitted = []
        while self.waiting:
            r = self.waiting[0]
            if self.active and self._used() + footprint(r, self.precision) > self.budget:
                break
            self.waiting.pop(0)
            r.admitted = self.clock()
            self.active.append(r)
            admitted.append(r)
        if admitted:
            keep = {}
            if self.union is not None:
                states = self.union.states(device=self.device_resident)
                t, _ = self.union.times()
                old = [r for r in self.active if r not in admitted]
                for i, r in enumerate(old):
                    keep[r.rid] = states[i]
                    keep[("t", r.rid)] = t[i]
            self._rebuild(keep)
        if not self.active:
            return False
        chunk = min(self.max_chunk, min(r.steps - r.done_steps for r in self.active))
        self.union.run(chunk)
        for r in self.active:
            r.done_steps += chunk
            K = np.array([1, 3, 6, 10, 15])[np.asarray(r.mesh["orders"], np.int64)]
            self.dof_stage_updates += chunk * self.kw["rk_order"] * 3 * int(K.sum())
        finished = [r for r in self.active if r.done_steps >= r.steps]
        if finished:
            states = self.union.states(device=self.device_resident)
            t, _ = self.union.times()
            now = self.clock()
            for i, r in enumerate(self.active):
                if r in finished:
                    r.result = states[i].cpu().numpy() if hasattr(states[i], "cpu") else states[i]
                    r.t_final = float(t[i])
                    r.finished = now
            keep = {}
            for i, r in enumerate(self.active):
                if r not in finished:
                    keep[r.rid] = states[i]
                    keep[("t", r.rid)] = t[i]
            self.active = [r for r in self.active if r not in finished]
            self.done.extend(finished)
            self._rebuild(keep)
        return True

    def run_until_idle(self):
        while self.step():
            pass

    def latencies(self):
        return np.array([r.finished - r.arrival for r in self.done])

    def close(self):
        if self.union is not None:
            self.union.close()
            self.union = None
