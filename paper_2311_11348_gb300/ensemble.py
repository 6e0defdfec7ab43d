"""Batched ensembles: several independent meshes in one libswedg context.

The members are concatenated into one disjoint-union mesh (vertex ids of
member m shifted by the vertices of members < m) and tagged with
swe_set_members, so every kernel of an RK stage is one launch over all
members while each member keeps its own CFL step and time.  This module only
concatenates and slices arrays; the arithmetic is in the CUDA library.
"""
from __future__ import annotations

import numpy as np

from . import swedg

KMAX = swedg.KMAX


class Ensemble:
    def __init__(self, members, **solver_kwargs):
        """members: list of dicts with xy [nv,2], tri [ne,3], hv [nv], orders [ne]
        and optionally bc_tag [ne,3]."""
        self.members = members
        self.nv = [len(m["xy"]) for m in members]
        self.ne = [len(m["tri"]) for m in members]
        self.v0 = np.concatenate([[0], np.cumsum(self.nv)]).astype(np.int64)
        self.e0 = np.concatenate([[0], np.cumsum(self.ne)]).astype(np.int64)
        xy = np.concatenate([m["xy"] for m in members]).astype(np.float64)
        tri = np.concatenate([np.asarray(m["tri"], np.int64) + self.v0[i] for i, m in enumerate(members)])
        hv = np.concatenate([m["hv"] for m in members]).astype(np.float64)
        orders = np.concatenate([np.asarray(m["orders"], np.int8) for m in members])
        tags = None
        if any(m.get("bc_tag") is not None for m in members):
            tags = np.concatenate([m["bc_tag"] if m.get("bc_tag") is not None else np.zeros((len(m["tri"]), 3), np.int8)
                                   for m in members]).astype(np.int8)
        member = np.concatenate([np.full(n, i, np.int32) for i, n in enumerate(self.ne)])
        self.solver = swedg.Solver(**solver_kwargs)
        self.solver.set_mesh(xy, tri.astype(np.int32), tags)
        self.solver.set_bathymetry(hv)
        self.solver.set_orders(orders)
        self.solver.set_members(len(members), member)

    @property
    def n(self):
        return len(self.members)

    def set_states(self, states, times=None):
        """states: per member c[3][15][ne_m], numpy (host) or torch CUDA tensors
        (device-resident: concatenated on the device, no host round trip)."""
        if all(hasattr(s, "is_cuda") and s.is_cuda for s in states):
            import torch
            c = torch.cat([s.to(torch.float64) for s in states], dim=2).contiguous()
            # the library reads on its own stream: wait for torch's stream only
            # (a device-wide sync would also wait for other contexts' steps)
            torch.cuda.current_stream().synchronize()
        else:
            c = np.zeros((3, KMAX, int(self.e0[-1])))
            for i, s in enumerate(states):
                c[:, :, self.e0[i]:self.e0[i + 1]] = s.cpu().numpy() if hasattr(s, "cpu") else s
        self.solver.set_state(c, 0.0)
        self.solver.set_member_times(np.zeros(self.n) if times is None else np.asarray(times, np.float64))

    def states(self, device=False):
        """per member c[3][15][ne_m]: numpy arrays, or torch CUDA tensors when device=True"""
        if device:
            import torch
            c = torch.empty((3, KMAX, int(self.e0[-1])), dtype=torch.float64, device="cuda")
            torch.cuda.current_stream().synchronize()  # the memory is free on torch's stream
            self.solver.get_state(c)  # written on the library's stream, complete on return
            return [c[:, :, self.e0[i]:self.e0[i + 1]].clone() for i in range(self.n)]
        c, _ = self.solver.get_state()
        return [c[:, :, self.e0[i]:self.e0[i + 1]].copy() for i in range(self.n)]

    def times(self):
        return self.solver.member_times()

    def member_status(self):
        """per member: the status bits its elements set since the last call (see swe_member_status)"""
        return self.solver.member_status()

    def run(self, nsteps, dt_fixed=0.0):
        self.solver.run(nsteps, dt_fixed)

    def close(self):
        self.solver.close()
