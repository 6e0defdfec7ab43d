#!/usr/bin/env python
"""Benchmark: DOF-stage updates/s of the SSP-RK3 step of the quadrature-free DG
shallow water scheme on the 131,072-triangle p-adaptive ocean workload
(256x256 split squares, +-20 % jitter, Fourier bathymetry 50..4000 m, orders
p in {1,2,3} at 70/20/10 %, CFL steps), FP64 and mixed precision, each with its
relative L2 error against the FP64 oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one SSP-RK3 step (3 stages) over the whole mesh; DOF-stage updates
per step = 3 stages x 3 fields x sum_e K(p_e).  The state (~40 MB in all RK
buffers) fits in the 129 MB L2, so L2 is flushed (256 MB write) between timed
steps and each step is timed alone with CUDA events on the solver's stream.
With N > 1 (torchrun), every rank runs an independent replica of the workload
(the path is replicas-only on this pool; no data-path collective).  The
default line also carries a short serving leg (p50/p99 completion latency).

Other workloads (one JSON line each):
    --workload ensemble   64 members, log-uniform 8k..600k triangles (9.3M in
                          all), p in {1..4}, one union context, per-member dt
    --workload serving    Poisson arrivals of such members (5k..200k
                          triangles, 100..500 steps by default), continuous
                          batching, p50/p99 latency and throughput
    --workload shelf      2,097,152 triangles, tanh shelf, M2 tide, p in {1..4}
    --workload sweep      the paper's statically adaptive p1-2 dam break
                          (2,097,152 triangles), fraction of p = 2 elements
                          0, 1/64, 1/32, 1/16, 1/8, 1; mixed and FP64
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2311_11348_gb300 import inputs  # noqa: E402

METRIC = "DOF-stage updates/s, mixed vs FP64 at stated L2 error; p50/p99 solve latency"
REPEATS, REPEAT_STEPS = 5, 34  # the median of 5 repeats of 34 SSP-RK3 steps (102 stages) each
ACC_STEPS = 100  # CFL steps of the accuracy comparison against the oracle
ADAPT = dict(up=0.05, down=1e-3, pmin=1, pmax=3, every=10, steps=100)  # the adaptive leg


def max_over_ranks(value, world, device="cuda"):
    """the maximum of a per-rank number over all ranks (the timed region's
    wall time of the slowest replica); the identity on one rank"""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, max_seconds):
    """whole-job throughput of N independent replicas: all ranks' units over the slowest rank's time"""
    return units_per_rank * world / max_seconds


def dofs_per_step(orders, stages=3):
    K = np.array([1, 3, 6, 10, 15])[orders.astype(np.int64)]
    return stages * 3 * int(K.sum())


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) > 2 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 2 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def single_mesh_workload(args):
    """the single-mesh workload of the run and its label"""
    if args.workload == "shelf":
        w = inputs.shelf_p1234(args.n_shelf)
        n = args.n_shelf
        return w, (f"shelf_p1234: {n}x{n} split squares ({2 * n * n} triangles), tanh shelf 4000 -> 20 m, "
                   f"M2 tide on x = 0, p in {{1..4}} 40/30/20/10, SSP-RK3, CFL 0.1")
    w = inputs.ocean_p123(args.n)
    return w, (f"ocean_p123: {args.n}x{args.n} split squares ({2 * args.n * args.n} triangles), "
               f"p in {{1,2,3}} 70/20/10, SSP-RK3, CFL 0.1")


def host_cpu():
    """(logical cores, CPU model) of this host, for the oracle baselines"""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return os.cpu_count() or 1, model or "unknown"


def oracle_mesh_params(w, threads=1):
    """the FP64 oracle on the workload's mesh; threads > 1 (0: every host core)
    runs its element loops on the threaded build of the same source"""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    tide = w.get("tide", (0.0, 0.0, 0.0))
    m = O.Mesh(w["xy"], w["tri"], w["hv"], w["orders"], bc_tag=w.get("bc_tag"), threads=threads)
    P = O.Params(g=w["g"], cfl=w["cfl"], rk_order=3, tide_amp=tide[0], tide_period=tide[1], tide_phase=tide[2])
    return m, P


def make_solver(w, precision, stream):
    from paper_2311_11348_gb300 import swedg
    s = swedg.Solver(g=w["g"], cfl=w["cfl"], rk_order=3, precision=precision, stream=stream,
                     tide=w.get("tide", (0.0, 0.0, 0.0)))
    s.set_mesh(w["xy"], w["tri"], w.get("bc_tag"))
    s.set_bathymetry(w["hv"])
    s.set_orders(w["orders"])
    return s


def initial_state(s, w):
    xi_v = w["ic"](w["xy"][:, 0], w["xy"][:, 1])[0]
    c = np.zeros((3, 15, len(w["tri"])))
    c[0, :3] = s.p1_modes(xi_v)
    return c


def run_ours(args, rank, world):
    import torch
    from paper_2311_11348_gb300 import swedg
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    w, _ = single_mesh_workload(args)
    ne = len(w["tri"])
    dps = dofs_per_step(w["orders"])
    stream = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    res = {}
    modes = {"mixed": swedg.PREC_MIXED_FP32, "fp64": swedg.PREC_FP64, "tf32": swedg.PREC_MIXED_TF32}
    order = [args.precision] + [k for k in ("mixed", "fp64", "tf32") if k != args.precision]
    prec_list = [(k, modes[k]) for k in order]
    clocks = None
    for name, prec in prec_list:
        s = make_solver(w, prec, stream.cuda_stream)
        c0 = initial_state(s, w)
        s.set_state(c0, 0.0)
        if args.shape:
            s.set_launch_shape(args.shape)
        shape = s.autotune(steps=5)[0] if args.autotune and not args.shape else s.launch_shape()
        s.run(args.warmup)
        s.set_state(c0, 0.0)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        if name == prec_list[0][0]:
            clocks = Clocks(int(os.environ.get("LOCAL_RANK", 0)))
        times = []
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                flush.add_(1.0)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                s.run(1)
                b.record(stream)
                times.append((a, b))
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in times]
        if name == prec_list[0][0]:
            clk = clocks.stop()
        tot = max_over_ranks(sum(ms), world)
        reps = None
        if name == prec_list[0][0]:  # 5 repeats of >= 100 stages each, for the median
            reps = []
            for _ in range(REPEATS):
                s.set_state(c0, 0.0)
                times = []
                with torch.cuda.stream(stream):
                    for _ in range(REPEAT_STEPS):
                        flush.add_(1.0)
                        a = torch.cuda.Event(enable_timing=True)
                        b = torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        s.run(1)
                        b.record(stream)
                        times.append((a, b))
                torch.cuda.synchronize()
                reps.append(max_over_ranks(sum(a.elapsed_time(b) for a, b in times), world) / REPEAT_STEPS)
        # per-family timing (separate profiled pass over the same steps)
        s.set_state(c0, 0.0)
        s.profile(True)
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                flush.add_(1.0)
                s.run(1)
        torch.cuda.synchronize()
        prof = s.profile_read()
        s.profile(True)
        s.set_state(c0, 0.0)
        s.run(args.steps)
        launches = s.profile_read()["kernels"][1]
        s.profile(False)
        res[name] = dict(ms_steps=ms, total_ms=tot, prof=prof, launches=launches, solver=s, c0=c0, shape=shape,
                         repeats=reps)
    return w, dps, res, clk, stream, flush


def accuracy(w, res, nsteps=100):
    """relative L2 error of every mode after nsteps CFL steps against the FP64
    oracle run from the same input (the threaded build, every host core)"""
    m, P = oracle_mesh_params(w, threads=0)
    out = {}
    c0 = res["fp64"]["c0"]
    t0 = time.perf_counter()
    c_o, t_o = m.run(P, c0, 0.0, nsteps)
    accuracy.oracle_s_per_step = (time.perf_counter() - t0) / nsteps
    for name in res:
        s = res[name]["solver"]
        s.set_state(c0, 0.0)
        s.run(nsteps)
        c_g, _ = s.get_state()
        out[name] = float(np.linalg.norm(c_g - c_o) / np.linalg.norm(c_o))
    return out, nsteps


def e2e_loop(s, hin, hout, steps, per_step=None):
    """every step: the state in from pinned host memory, one SSP-RK3 step, the
    state out to pinned host memory (packed layout), through the asynchronous
    C ABI calls (copies double-buffered on copy streams, overlapping the
    previous / next step); one swe_sync at the end.  Returns the wall time."""
    import torch
    s.set_state_packed_async(hin, 0.0)
    s.run_async(1)
    s.get_state_packed_async(hout[0])
    s.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        s.set_state_packed_async(hin, 0.0)
        if per_step is not None:
            per_step()
        s.run_async(1)
        s.get_state_packed_async(hout[k % 2])
    s.sync()
    return time.perf_counter() - t0


def e2e(w, res, name, steps, stream):
    """the same step through the C ABI with pinned host buffers: state in, one
    step, state out (host<->device copies inside the timed region), in the
    packed state layout (the modes each element's order has)"""
    import torch
    s = res[name]["solver"]
    s.set_state(res[name]["c0"], 0.0)
    hin = torch.from_numpy(s.get_state_packed()[0]).pin_memory()
    hout = [torch.empty_like(hin).pin_memory() for _ in range(2)]
    dt = e2e_loop(s, hin, hout, steps)
    nbytes = hin.numel() * 8
    return dt, nbytes


def oracle_rate(w, steps, warmup, threads=1):
    """seconds of `steps` full-mesh RK3 steps of the FP64 oracle on the
    workload (after `warmup` untimed ones); threads as in oracle_mesh_params"""
    m, P = oracle_mesh_params(w, threads=threads)
    xi_v = w["ic"](w["xy"][:, 0], w["xy"][:, 1])[0]
    c = np.zeros((3, 15, len(w["tri"])))
    c[0, :3] = m.p1_modes(xi_v)
    for _ in range(warmup):
        c, _, _ = m.step(P, c, 0.0)
    t0 = time.perf_counter()
    t = 0.0
    for _ in range(steps):
        c, t, _ = m.step(P, c, t)
    return time.perf_counter() - t0


def adaptive_leg(w, res, stream):
    """The adaptive run of the workload's recipe: ADAPT["steps"] SSP-RK3 CFL
    steps with the modal-decay indicator every ADAPT["every"] steps (orders in
    ADAPT["pmin"]..ADAPT["pmax"]), FP64 and mixed mode side by side from the
    same initial state.  The FP64 context takes the decisions (swe_adapt) and
    the mixed context is given the same order map, so that the two states are
    compared on one trajectory of maps; reported: their relative L2 distance
    at the end, and the wall time of one adaptation (indicator, order change
    and the rebuild of the context's device description it triggers)."""
    import torch
    c0 = res["fp64"]["c0"]
    ctx = {}
    for name in ("fp64", "mixed"):
        s = make_solver(w, {"fp64": 0, "mixed": 1}[name], stream.cuda_stream)
        s.set_launch_shape(res[name]["shape"])
        s.set_state(c0, 0.0)
        ctx[name] = s
    a = ADAPT
    adapt_s, changed = [], []
    for _ in range(a["steps"] // a["every"]):
        for s in ctx.values():
            s.run(a["every"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        orders, n = ctx["fp64"].adapt(a["up"], a["down"], a["pmin"], a["pmax"])
        ctx["fp64"].packed_size()  # the rebuild the order change triggers
        adapt_s.append(time.perf_counter() - t0)
        changed.append(n)
        ctx["mixed"].set_orders(orders)
    cf, tf = ctx["fp64"].get_state()
    cm, tm = ctx["mixed"].get_state()
    for s in ctx.values():
        s.close()
    return {"steps": a["steps"], "adapt_every": a["every"], "theta_up": a["up"], "theta_down": a["down"],
            "orders": [a["pmin"], a["pmax"]],
            "mixed_vs_fp64_rel_l2": float(np.linalg.norm(cm - cf) / np.linalg.norm(cf)),
            "t_end_s": tf, "adapt_ms_mean": 1e3 * float(np.mean(adapt_s)), "adapt_ms_max": 1e3 * float(np.max(adapt_s)),
            "changed_per_pass_mean": float(np.mean(changed)),
            "final_order_counts": np.bincount(orders, minlength=5)[1:4].tolist()}


def ensemble_state(ens, members):
    """initial union state: P1 interpolant of each member's vertex elevation, momenta at rest"""
    xi = np.concatenate([m["xi_vertex"] for m in members])
    c = np.zeros((3, 15, int(ens.e0[-1])))
    c[0, :3] = ens.solver.p1_modes(xi)
    return c


def bench_ensemble(args, world):
    """Batched ensemble: every member in one union context; each timed step is
    one SSP-RK3 step of all members (graph replay), every member at its own
    CFL step."""
    import torch
    from paper_2311_11348_gb300 import ensemble, swedg
    members = inputs.ensemble_members(args.members)
    orders = np.concatenate([m["orders"] for m in members])
    dps = dofs_per_step(orders)
    stream = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    res = {}
    clk = None
    small = int(np.argmin([len(m["tri"]) for m in members]))
    for name, prec in [("mixed", swedg.PREC_MIXED_FP32), ("fp64", swedg.PREC_FP64), ("tf32", swedg.PREC_MIXED_TF32)]:
        t_build = time.perf_counter()
        ens = ensemble.Ensemble(members, g=9.81, cfl=0.1, rk_order=3, precision=prec, stream=stream.cuda_stream)
        c0 = ensemble_state(ens, members)
        t_build = time.perf_counter() - t_build
        ens.solver.set_state(c0, 0.0)
        shape = ens.solver.autotune(steps=2)[0] if args.autotune else ens.solver.launch_shape()
        ens.run(args.warmup)
        ens.solver.set_state(c0, 0.0)
        ens.solver.set_member_times(np.zeros(ens.n))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        if clk is None:
            clocks = Clocks(int(os.environ.get("LOCAL_RANK", 0)))
        times = []
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                flush.add_(1.0)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ens.run(1)
                b.record(stream)
                times.append((a, b))
        torch.cuda.synchronize()
        if clk is None:
            clk = clocks.stop()
        tot = max_over_ranks(sum(a.elapsed_time(b) for a, b in times), world)
        ens.solver.set_state(c0, 0.0)
        ens.solver.set_member_times(np.zeros(ens.n))
        ens.solver.profile(True)
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                flush.add_(1.0)
                ens.run(1)
        torch.cuda.synchronize()
        prof = ens.solver.profile_read()
        ens.solver.profile(True)
        ens.solver.set_state(c0, 0.0)
        ens.solver.set_member_times(np.zeros(ens.n))
        ens.run(args.steps)
        launches = ens.solver.profile_read()["kernels"][1]
        ens.solver.profile(False)
        err = None
        if not args.no_oracle:  # the smallest member after 2 of its own CFL steps, against the oracle
            sys.path.insert(0, os.path.join(ROOT, "oracle"))
            import oracle as O
            ens.solver.set_state(c0, 0.0)
            ens.solver.set_member_times(np.zeros(ens.n))
            ens.run(2)
            got = ens.states()[small]
            m = members[small]
            om = O.Mesh(m["xy"], m["tri"], m["hv"], m["orders"])
            ref, _ = om.run(O.Params(g=9.81, cfl=0.1, rk_order=3), c0[:, :, ens.e0[small]:ens.e0[small + 1]], 0.0, 2)
            err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        e2e_rate = e2e_bytes = None
        if name == "mixed":  # end to end through the API: pinned host state in (packed), one step, state out
            ens.solver.set_state(c0, 0.0)
            hin = torch.from_numpy(ens.solver.get_state_packed()[0]).pin_memory()
            hout = [torch.empty_like(hin).pin_memory() for _ in range(2)]
            n_e2e = 5
            e2e_rate = dps * n_e2e / e2e_loop(ens.solver, hin, hout, n_e2e)
            e2e_bytes = hin.numel() * 8
            del hin, hout
        res[name] = dict(total_ms=tot, prof=prof, launches=launches, err=err, build_s=t_build,
                         bytes=ens.solver.memory_bytes(), shape=shape, e2e=e2e_rate, e2e_bytes=e2e_bytes)
        ens.close()
    value = job_rate(dps * args.steps, world, res["mixed"]["total_ms"] / 1e3)
    fp64 = job_rate(dps * args.steps, world, res["fp64"]["total_ms"] / 1e3)
    tf32 = job_rate(dps * args.steps, world, res["tf32"]["total_ms"] / 1e3)
    fams = {k: v for k, v in res["mixed"]["prof"].items() if k != "kernels"}
    dom = max(fams, key=lambda k: fams[k][0])
    ne = len(orders)
    w = dict(orders=orders)
    line = {
        "metric": METRIC, "value": value, "unit": "DOF-stage/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["mixed"]["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": f"ensemble: {len(members)} members, log-uniform {ne // len(members)} mean "
                               f"({min(len(m['tri']) for m in members)}..{max(len(m['tri']) for m in members)}) "
                               f"triangles, {ne} in all, p in {{1..4}} 40/30/20/10, SSP-RK3, CFL 0.1, per-member dt",
                   "members": len(members), "triangles": ne, "dof_stage_per_step": dps, "precision": "mixed",
                   "l2": "inputs larger than L2; 256 MB flush between timed steps", "replicas": world},
        "mixed": {"value": value, "rel_l2_vs_oracle": res["mixed"]["err"], "oracle_member_triangles":
                  len(members[small]["tri"]), "oracle_steps": 2, "device_bytes": res["mixed"]["bytes"],
                  "setup_s": res["mixed"]["build_s"], "launch_shape": res["mixed"]["shape"]},
        "fp64": {"value": fp64, "ms_per_step": res["fp64"]["total_ms"] / args.steps,
                 "rel_l2_vs_oracle": res["fp64"]["err"], "device_bytes": res["fp64"]["bytes"],
                 "launch_shape": res["fp64"]["shape"]},
        "tf32": {"value": tf32, "ms_per_step": res["tf32"]["total_ms"] / args.steps,
                 "rel_l2_vs_oracle": res["tf32"]["err"], "device_bytes": res["tf32"]["bytes"],
                 "launch_shape": res["tf32"]["shape"],
                 "kernel_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in res["tf32"]["prof"].items()
                                        if k != "kernels"}},
        "mixed_over_fp64": value / fp64,
        "tf32_over_fp64": tf32 / fp64,
        "kernel_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in fams.items()},
        "dominant_kernel": dom, "gpu_launches": int(res["mixed"]["launches"]), "clocks": clk,
        "e2e": {"value": res["mixed"]["e2e"] * world, "unit": "DOF-stage/s",
                "h2d_bytes_per_step": res["mixed"]["e2e_bytes"], "d2h_bytes_per_step": res["mixed"]["e2e_bytes"]},
    }
    line["roofline"] = roofline(w, res["mixed"], dom, args.steps, peaks(), "mixed")
    return line


def serving_run(rate, duration, tri_lo, tri_hi, steps_lo, steps_hi, budget_gb, chunk, warmup, seed=7, pool=0,
                drain_s=None):
    """Continuous-batching serving loop against a wall clock: requests arrive
    by a seeded Poisson process over `duration` seconds, are admitted by
    device footprint, share RK launches with the running ones and leave when
    done.  pool > 0 draws the requests' meshes from that many pre-generated
    members (see inputs.serving_requests).  The loop ends when every request
    is done, or drain_s seconds after the last arrival (then the unfinished
    ones are the backlog).  Returns a summary."""
    import torch
    from paper_2311_11348_gb300 import serve, swedg
    reqs = inputs.serving_requests(rate, duration, tri_lo, tri_hi, steps_lo, steps_hi, seed=seed, pool=pool)
    prepared, initial = [], {}
    for k, (t_arr, m, steps) in enumerate(reqs):  # client side: initial states, before the clock starts
        if id(m) not in initial:
            s = swedg.Solver()
            s.set_mesh(m["xy"], m["tri"])
            c = np.zeros((3, 15, len(m["tri"])))
            c[0, :3] = s.p1_modes(m["xi_vertex"])
            s.close()
            initial[id(m)] = c
        mesh = dict(xy=m["xy"], tri=m["tri"], hv=m["hv"], orders=m["orders"])
        prepared.append((t_arr, serve.Request(rid=k, mesh=mesh, state=initial[id(m)], steps=steps)))
    kw = dict(precision=swedg.PREC_MIXED_FP32, g=9.81, cfl=0.1, rk_order=3, max_chunk=chunk)
    # warm-up: one small request through the same path (module load, graph capture)
    srv = serve.Server(int(budget_gb * 1e9), **kw)
    w0 = min((r for _, r in prepared), key=lambda r: len(r.mesh["tri"]))
    srv.submit(serve.Request(rid=-1, mesh=w0.mesh, state=w0.state, steps=max(3, warmup), arrival=1.0))
    srv.run_until_idle()
    srv.close()
    torch.cuda.synchronize()
    srv = serve.Server(int(budget_gb * 1e9), **kw)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", 0)))
    t0 = time.perf_counter()
    pending = list(prepared)
    busy = 0.0
    stop = None if drain_s is None else duration + drain_s
    occ = []  # (time, requests in the system: admitted or waiting) at every scheduling point
    while pending or srv.waiting or srv.in_flight:
        now = time.perf_counter() - t0
        occ.append((now, len(srv.waiting) + len(srv.in_flight)))
        if stop is not None and now >= stop:
            break
        while pending and pending[0][0] <= now:
            t_arr, r = pending.pop(0)
            r.arrival = t0 + t_arr
            srv.submit(r)
        if not srv.waiting and not srv.in_flight:
            time.sleep(max(0.0, min(0.05, pending[0][0] - now)))
            continue
        tb = time.perf_counter()
        srv.step()
        busy += time.perf_counter() - tb
    makespan = time.perf_counter() - t0
    clk = clocks.stop()
    backlog = len(pending) + len(srv.waiting) + len(srv.in_flight)
    srv.close()
    lat = srv.latencies()
    arr = np.array([r.arrival - t0 for r in srv.done])
    work = srv.dof_stage_updates
    offered = sum(r.steps * 3 * 3 * int(np.array([1, 3, 6, 10, 15])[r.mesh["orders"].astype(np.int64)].sum())
                  for _, r in prepared) / duration
    state_bytes = sum(r.state.nbytes for _, r in prepared)
    pct = (lambda a, q: float(np.percentile(a, q)) if len(a) else None)
    first, second = lat[arr < duration / 2], lat[(arr >= duration / 2) & (arr < duration)]
    p99a, p99b = pct(first, 99), pct(second, 99)
    # requests in the system, time-averaged over each half of the arrival window
    def occupancy(lo, hi):
        acc = span = 0.0
        for (ta, na), (tb, _) in zip(occ, occ[1:]):
            a, b = max(ta, lo), min(tb, hi)
            if b > a:
                acc += na * (b - a)
                span += b - a
        return acc / span if span > 0 else None
    occ_a, occ_b = occupancy(0.0, duration / 2), occupancy(duration / 2, duration)
    # stable: the server keeps up with the arrivals -- every request of the
    # window done, within a tenth of the window after the last arrival.  The
    # request sizes span three decades (the largest take ~20 s alone), so the
    # p99 of a half window is its slowest request or two and the number of
    # requests in the system follows when the largest ones arrive: both are
    # reported, not used for the decision.
    stable = backlog == 0 and makespan - duration <= 0.1 * duration
    return dict(value=work / makespan, requests=len(prepared), completed=len(srv.done), backlog=backlog,
                failed=len(srv.failed), makespan_s=makespan, rate=rate,
                p50_s=pct(lat, 50), p99_s=pct(lat, 99), mean_s=float(lat.mean()) if len(lat) else None,
                max_s=float(lat.max()) if len(lat) else None, p99_first_half_s=p99a, p99_second_half_s=p99b,
                in_system_first_half=occ_a, in_system_second_half=occ_b,
                stable=stable, offered_dof_stage_per_s=offered,
                dof_stage_updates=work, rebuilds=srv.rebuilds, rebuild_s=srv.rebuild_s, busy_s=busy,
                launches=srv.launches, state_bytes=state_bytes,
                total_steps=sum(r.steps for _, r in prepared),
                mean_triangles=float(np.mean([len(r.mesh["tri"]) for _, r in prepared])), clocks=clk)


def bench_sweep(args, world):
    """The paper's statically adaptive p1-2 study (Sect. 5, radial dam break on
    a perturbed uniform mesh of 2,097,152 triangles): every nth element at p = 2,
    fractions 0, 1/64, 1/32, 1/16, 1/8, 1; mixed and FP64 modes, each with the
    autotuned launch shape (--shape: that one; --no-autotune: the default), W
    warm-up and K timed steps each (CUDA events, L2 flushed)."""
    import torch
    from paper_2311_11348_gb300 import swedg
    stream = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    n = args.n_shelf
    rows = []
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", 0)))
    for nth, frac in ((0, "0"), (64, "1/64"), (32, "1/32"), (16, "1/16"), (8, "1/8"), (1, "1")):
        w = inputs.dam_break_p12(n, nth)
        dps = dofs_per_step(w["orders"])
        row = {"fraction_p2": frac, "triangles": len(w["tri"]), "dof_stage_per_step": dps}
        for name, prec in (("mixed", swedg.PREC_MIXED_FP32), ("fp64", swedg.PREC_FP64)):
            s = make_solver(w, prec, stream.cuda_stream)
            c0 = initial_state(s, w)
            s.set_state(c0, 0.0)
            if args.shape:
                s.set_launch_shape(args.shape)
            elif args.autotune:
                s.autotune(steps=2)
            row[name + "_launch_shape"] = list(s.launch_shape())
            s.set_state(c0, 0.0)
            s.run(args.warmup)
            torch.cuda.synchronize()
            times = []
            with torch.cuda.stream(stream):
                for _ in range(args.steps):
                    flush.add_(1.0)
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    s.run(1)
                    b.record(stream)
                    times.append((a, b))
            torch.cuda.synchronize()
            tot = max_over_ranks(sum(a.elapsed_time(b) for a, b in times), world)
            row[name] = {"value": job_rate(dps * args.steps, world, tot / 1e3),
                         "ms_per_stage": tot / args.steps / 3.0}
            s.close()
        rows.append(row)
    clk = clocks.stop()
    head = next(r for r in rows if r["fraction_p2"] == "1/32")
    return {"metric": METRIC, "value": head["mixed"]["value"], "unit": "DOF-stage/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 3.0 * head["mixed"]["ms_per_stage"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic",
            "config": {"workload": f"dam break p1-2 sweep: {n}x{n} perturbed split squares ({2 * n * n} triangles), "
                                   "flat 10 m bottom, radial dam, walls, every nth element at p = 2; value = the mixed "
                                   "mode at 1/32", "l2": "flushed between timed steps (256 MB write)", "replicas": world,
                       "launch_shape": list(args.shape) if args.shape else ("autotuned per fraction and mode"
                                                                             if args.autotune else "default")},
            "sweep": rows, "clocks": clk}


def bench_serving(args, world):
    """The serving loop at one offered rate (--rate), and with --rates a
    sweep of rates for the highest one whose p99 stays stable."""
    def one(rate):
        r = serving_run(rate, args.duration, args.tri_lo, args.tri_hi, args.steps_lo, args.steps_hi,
                        args.budget_gb, args.chunk, args.warmup, pool=args.pool, drain_s=args.drain_s)
        r["makespan_s"] = max_over_ranks(r["makespan_s"], world)
        r["value"] = r["dof_stage_updates"] / r["makespan_s"]
        return r
    r = one(args.rate)
    sweep = [one(x) for x in args.rates] if args.rates else []
    stable = [x["rate"] for x in [r] + sweep if x["stable"]]
    pool = f", meshes drawn from a pool of {args.pool} seeded members" if args.pool else ""
    drain = (f"; the loop stops {args.drain_s} s after the last arrival (unfinished requests: backlog)"
             if args.drain_s is not None else "; every request runs to completion")
    line = {
        "metric": METRIC, "value": r["value"] * world, "unit": "DOF-stage/s", "n_gpus": world,
        "steps": r["total_steps"], "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": f"serving: Poisson arrivals {args.rate}/s for {args.duration} s, triangles "
                               f"log-uniform [{int(args.tri_lo)}, {int(args.tri_hi)}], steps uniform "
                               f"[{args.steps_lo}, {args.steps_hi}], p in {{1..4}} 40/30/20/10, mixed, "
                               f"{args.budget_gb} GB admission budget, chunks of <= {args.chunk} steps{pool}{drain}",
                   "requests": r["requests"], "mean_triangles": r["mean_triangles"], "replicas": world,
                   "l2": "wall clock, end to end (state in from host, result out to host)"},
        "latency_s": {"p50": r["p50_s"], "p99": r["p99_s"], "mean": r["mean_s"], "max": r["max_s"],
                      "p99_first_half": r["p99_first_half_s"], "p99_second_half": r["p99_second_half_s"]},
        "completed": r["completed"], "backlog": r["backlog"], "failed": r["failed"],
        "in_system": {"first_half": r["in_system_first_half"], "second_half": r["in_system_second_half"]},
        "offered_dof_stage_per_s": r["offered_dof_stage_per_s"],
        "makespan_s": r["makespan_s"], "rebuilds": r["rebuilds"], "rebuild_s": r["rebuild_s"],
        "gpu_launches": r["launches"], "clocks": r["clocks"],
        "e2e": {"value": r["value"] * world, "unit": "DOF-stage/s",
                "h2d_bytes_per_step": r["state_bytes"] / max(r["total_steps"], 1),
                "d2h_bytes_per_step": r["state_bytes"] / max(r["total_steps"], 1)},
        "roofline": None,
    }
    if sweep:
        line["rate_sweep"] = sorted(({k: x[k] for k in ("rate", "requests", "completed", "backlog", "p50_s", "p99_s",
                                                       "p99_first_half_s", "p99_second_half_s", "in_system_first_half",
                                                       "in_system_second_half", "stable", "value",
                                                       "offered_dof_stage_per_s", "makespan_s", "rebuild_s")}
                                     for x in [r] + sweep), key=lambda x: x["rate"])
        line["highest_stable_rate_per_s"] = max(stable) if stable else None
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "tf32"],
                    help="headline mode: FP32 correction, FP64 throughout, or tensor-core (TF32 x3) correction")
    ap.add_argument("--n", type=int, default=256, help="split-square grid size (256: 131,072 triangles)")
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle accuracy and cpu_baseline legs")
    ap.add_argument("--workload", default="ocean", choices=["ocean", "shelf", "ensemble", "serving", "sweep"])
    ap.add_argument("--n-shelf", type=int, default=1024, help="shelf workload grid size (1024: 2,097,152 triangles)")
    ap.add_argument("--members", type=int, default=64, help="ensemble members")
    ap.add_argument("--rate", type=float, default=4.0, help="serving: arrivals per second")
    ap.add_argument("--duration", type=float, default=30.0, help="serving: seconds of arrivals")
    ap.add_argument("--tri-lo", type=float, default=5e3)
    ap.add_argument("--tri-hi", type=float, default=2e5)
    ap.add_argument("--steps-lo", type=int, default=100)
    ap.add_argument("--steps-hi", type=int, default=500)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--chunk", type=int, default=50, help="serving: max steps between scheduling points")
    ap.add_argument("--pool", type=int, default=0, help="serving: draw the meshes from this many members (0: one each)")
    ap.add_argument("--drain-s", type=float, default=None,
                    help="serving: stop this long after the last arrival (default: run every request to completion)")
    ap.add_argument("--rates", type=lambda v: [float(x) for x in v.split(",")], default=None,
                    help="serving: also sweep these arrival rates for the highest stable one")
    ap.add_argument("--no-serving", action="store_true", help="skip the short serving leg of the ocean workload")
    ap.add_argument("--no-adaptive", action="store_true", help="skip the adaptive leg of the ocean workload")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default launch shape instead of autotuning it per mode")
    ap.add_argument("--shape", type=lambda v: tuple(int(x) for x in v.split(",")), default=None,
                    help="launch shape to use instead of the autotuner's (6 comma-separated integers, see swedg.h)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    workload = single_mesh_workload(args)[1] if args.workload in ("ocean", "shelf") else args.workload

    def config_of(w, replicas):
        """the workload's config, the same dict in both arms"""
        return {"workload": workload, "triangles": len(w["tri"]), "dof_stage_per_step": dofs_per_step(w["orders"]),
                "l2": "GPU arm: flushed between timed steps (256 MB write)", "replicas": replicas}

    if args.impl == "reference":
        if rank != 0:
            return
        # every step a bounded sample of the workload: the same recipe, on the
        # full grid unless the W warm-up and K timed steps of the threaded
        # oracle (every host core) would take more than about two minutes
        # (cost per element-step calibrated on 32x32), else on a smaller grid
        import copy
        sys.path.insert(0, os.path.join(ROOT, "oracle"))
        import oracle as O
        threads = O.threaded(0)
        cores, model = host_cpu()
        steps, warm = max(1, args.steps), max(0, args.warmup)
        n_full = args.n_shelf if args.workload == "shelf" else args.n
        probe = copy.copy(args)
        probe.n = probe.n_shelf = 32
        wp, _ = single_mesh_workload(probe)
        per_elem = oracle_rate(wp, 2, 1, threads=0) / 2 / len(wp["tri"])
        n = n_full
        while n > 32 and per_elem * 2 * n * n * (steps + warm) > 120.0:
            n //= 2
        sample = copy.copy(args)
        sample.n = sample.n_shelf = n
        w, _ = single_mesh_workload(sample)
        sec = oracle_rate(w, steps, warm, threads=0)
        dps = dofs_per_step(w["orders"])
        v = dps * steps / sec
        what = "the full workload" if n == n_full else f"the same recipe at {n}x{n}"
        w_full = single_mesh_workload(args)[0] if n != n_full else w
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DOF-stage/s", "n_gpus": args.gpus,
                "steps": steps, "warmup": warm, "ms_per_step": 1e3 * sec / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config_of(w_full, args.gpus),
                "cpu_baseline": {"value": v, "unit": "DOF-stage/s", "cores": threads, "kind": "oracle",
                                 "nproc": cores, "cpu_model": model,
                                 "sample": f"{steps} SSP-RK3 steps (after {warm} warm-up steps) of the FP64 C oracle, "
                                           f"threaded build ({threads} OpenMP threads over elements), on {what} "
                                           f"({len(w['tri'])} triangles)"},
                "e2e": {"value": v, "unit": "DOF-stage/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    if args.workload in ("ensemble", "serving", "sweep"):
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        line = {"ensemble": bench_ensemble, "serving": bench_serving, "sweep": bench_sweep}[args.workload](args, world)
        if rank == 0:
            print(json.dumps(line))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    w, dps, res, clk, stream, flush = run_ours(args, rank, world)
    head = args.precision
    others = [k for k in res if k != head]
    acc, acc_steps = ({}, 0) if args.no_oracle else accuracy(w, res, nsteps=2 if args.workload == "shelf" else ACC_STEPS)
    value = job_rate(dps * args.steps, world, res[head]["total_ms"] / 1e3)
    rate = {k: job_rate(dps * args.steps, world, res[k]["total_ms"] / 1e3) for k in res}
    e2e_steps = max(5, args.steps)
    e2e_s, e2e_bytes = e2e(w, res, head, e2e_steps, stream)
    e2e_s = max_over_ranks(e2e_s, world)
    pk = peaks()
    # dominant kernel family of the headline mode (profiled pass)
    prof = res[head]["prof"]
    fams = {k: v for k, v in prof.items() if k != "kernels"}
    dom = max(fams, key=lambda k: fams[k][0])
    line = {
        "metric": METRIC, "value": value, "unit": "DOF-stage/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res[head]["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"mixed": "f64+f32", "fp64": "f64", "tf32": "f64+f32+tf32"}[head],
        "data": "synthetic",
        "config": config_of(w, world),
        "precision": head,
        "modes": {k: {"value": rate[k], "ms_per_step": res[k]["total_ms"] / args.steps,
                      "rel_l2_vs_oracle": acc.get(k), "oracle_steps": acc_steps,
                      "launch_shape": res[k]["shape"]} for k in res},
        "mixed_over_fp64": rate["mixed"] / rate["fp64"],
        "tf32_over_fp64": rate["tf32"] / rate["fp64"],
        "repeats": {"n": REPEATS, "steps_each": REPEAT_STEPS, "stages_each": 3 * REPEAT_STEPS,
                    "ms_per_step_median": statistics.median(res[head]["repeats"]),
                    "ms_per_step_min": min(res[head]["repeats"]), "ms_per_step_max": max(res[head]["repeats"]),
                    "value_median": job_rate(dps, world, statistics.median(res[head]["repeats"]) / 1e3)},
        "kernel_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in fams.items()},
        "dominant_kernel": dom,
        "gpu_launches": int(res[head]["launches"]),
        "clocks": clk,
        "e2e": {"value": dps * e2e_steps * world / e2e_s, "unit": "DOF-stage/s",
                "h2d_bytes_per_step": e2e_bytes, "d2h_bytes_per_step": e2e_bytes},
    }
    line["roofline"] = roofline(w, res[head], dom, args.steps, pk, head)
    if not args.no_serving and args.workload == "ocean":
        r = serving_run(rate=3.0, duration=8.0, tri_lo=5e3, tri_hi=1e5, steps_lo=100, steps_hi=300, budget_gb=150.0,
                        chunk=50, warmup=args.warmup)
        line["serving"] = {"p50_s": r["p50_s"], "p99_s": r["p99_s"], "value": r["value"], "unit": "DOF-stage/s",
                           "requests": r["requests"], "offered_dof_stage_per_s": r["offered_dof_stage_per_s"],
                           "rebuild_s": r["rebuild_s"], "makespan_s": r["makespan_s"],
                           "workload": "Poisson 3/s for 8 s, triangles log-uniform [5k, 100k], steps U[100, 300], "
                                       "p in {1..4} 40/30/20/10, mixed, wall clock end to end"}
    if args.workload == "ocean" and not args.no_adaptive:
        line["adaptive"] = adaptive_leg(w, res, stream)
    if rank == 0 and not args.no_oracle:
        # the threaded oracle on every host core (the large shelf mesh reuses
        # the timing of the accuracy check), and one step single-threaded
        import oracle as O
        threads = O.threaded(0)
        cores, model = host_cpu()
        if args.workload == "shelf":
            sec_n, n_steps = accuracy.oracle_s_per_step, 1
        else:
            n_steps = 3
            sec_n = oracle_rate(w, n_steps, 1, threads=0) / n_steps
        sec_1 = oracle_rate(w, 1, 0, threads=1)
        line["cpu_baseline"] = {"value": dps / sec_n, "unit": "DOF-stage/s", "cores": threads, "kind": "oracle",
                                "nproc": cores, "cpu_model": model,
                                "sample": f"{n_steps} full-mesh SSP-RK3 steps of the FP64 C oracle, threaded build "
                                          f"({threads} OpenMP threads over elements)",
                                "single_core": {"value": dps / sec_1, "cores": 1,
                                                "sample": "1 full-mesh SSP-RK3 step of the serial build"}}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


# DRAM bytes (read + write) per launch of the base kernels on the 131,072-
# triangle ocean workload with the autotuned ocean shape (uncapped base grids:
# the 128-register element kernel), from one ncu capture of the current
# kernels (cold cache), TRAFFIC_CAPTURE below, run after the same command
# exited 0 without ncu: the mean over an SSP-RK3 step's launches (the element
# kernel reads the step's start state in two of the three stages).  None for
# other workloads and kernels.
MEASURED_TRAFFIC = {"edge_base": (41.240832e6 + 0.227584e6 + 41.236480e6 + 0.071680e6) / 2.0,
                    "elem_base": ((62.336256e6 + 0.406528e6) + 2.0 * (71.815936e6 + 0.165376e6)) / 3.0}
TRAFFIC_CAPTURE = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control "
                   "none -k regex:'k_edge_base|k_elem_base' -s 6 -c 4 python bench.py --steps 2 --warmup 3 --no-oracle "
                   "--no-serving --no-adaptive --shape 0,128,128,64,1,2")


def roofline(w, r, dom, steps, pk, head):
    """Roofline of the dominant kernel family: algorithmic flops per launch
    (roofline.py) over the family's mean CUDA-event time per launch (profiled
    pass), against the peak of the pipe that bounds it (FP64 for the base
    kernels and the FP64 mode, FP32 for the mixed-mode correction)."""
    from paper_2311_11348_gb300 import roofline as rl
    ms, n = r["prof"][dom]
    if n == 0:
        return None
    f = rl.family_flops(w["orders"], dom, mode=head)
    if f is None:
        return None
    per_launch_s = ms / n / 1e3
    launches_per_step = n / steps
    achieved = f / launches_per_step / per_launch_s / 1e12
    pipe = rl.pipe_of(dom, head)
    if pipe == "tensor":
        bf16 = pk.get("bf16_tflops_sustained")
        peak = bf16 * rl.TF32_OVER_BF16 if bf16 else 1700.0 * rl.TF32_OVER_BF16
        note = ("dense TF32 = measured sustained BF16 (MEASURED_PEAKS.json) x 1.1/2.25 (nominal ratio)" if bf16
                else "dense TF32 = fallback 1.7 PFLOP/s sustained BF16 x 1.1/2.25")
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": dom, "pipe": pipe, "flops_per_step": f, "peak_source": note}
    peak = rl.FP64_PEAK_TFLOPS if pipe == "fp64" else rl.FP32_PEAK_TFLOPS
    note = ("FP64 pipe, 152 SMs x 4 flop/clk x 2.07 GHz (nominal; measured DFMA loop 1.19 TFLOP/s at 1.92 GHz)"
            if pipe == "fp64" else "FP32 pipe, 152 SMs x 256 flop/clk x 2.07 GHz (nominal; measured FFMA loop 74.6 "
            "TFLOP/s at 1.92 GHz)")
    traffic = MEASURED_TRAFFIC.get(dom) if len(w["orders"]) == 131072 and pipe == "fp64" else None
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": traffic, "kernel": dom, "pipe": pipe, "flops_per_step": f, "peak_source": note}
    if traffic is not None:
        out["traffic_source"] = TRAFFIC_CAPTURE
    return out


if __name__ == "__main__":
    main()
