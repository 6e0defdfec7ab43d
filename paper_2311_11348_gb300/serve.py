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
# device bytes per element of a union context, measured from swe_memory_bytes
# of representative meshes (state x3, velocity, fluxes, geometry, staging)
BYTES_PER_ELEMENT_FP64 = 2600
BYTES_PER_ELEMENT_MIXED = 2200


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


def footprint(req: Request, precision: int) -> int:
    per = BYTES_PER_ELEMENT_MIXED if precision == swedg.PREC_MIXED_FP32 else BYTES_PER_ELEMENT_FP64
    return per * len(req.mesh["tri"])


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
