"""Continuous-batching server for gradient evaluations (serving workload).

Requests of different grid sizes from concurrent optimisations arrive at any time.  The
dispatcher admits a waiting request as soon as a slot is free and its device footprint
(``fdtd_footprint_bytes``) fits the remaining HBM budget; every admitted request owns a handle
(fields, CPML state, pole currents and DFTs resident on the device) and its own CUDA stream, and
runs its forward / adjoint / gradient as captured CUDA graphs of 16 time steps.  Requests on the
device therefore overlap: the GPU's hardware scheduler interleaves the blocks of every stream's
graphs, which fills the 152 SMs even with grids (48^3 ... 192^3) too small to do it alone.
Finished requests release their slot and memory immediately, and the next waiting request is
admitted (continuous batching, FIFO among the waiting).

Each result is bitwise independent of the mix: a request's state is private and every kernel is
deterministic (no cross-request reductions or atomics on data).
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time

import numpy as np

from . import _native as N
from .problem import Problem


class Request:
    """One gradient evaluation: grid description, materials, density (host array)."""

    def __init__(self, desc, bg, m1, m2, rho, gamma=0.0, rid=None, t_arrival=None, t_arrival_rel=0.0):
        self.desc, self.bg, self.m1, self.m2, self.rho, self.gamma = desc, bg, m1, m2, rho, gamma
        self.id = rid
        self.t_arrival = t_arrival
        self.t_arrival_rel = t_arrival_rel      # offset in the replayed stream (s)
        self.poles_total = [len(m1["poles"][k]) + len(m2["poles"][k]) for k in range(3)]

    def footprint(self):
        return N.fdtd_footprint_bytes(self.desc, self.poles_total)

    def cell_updates(self):
        d = self.desc
        return 2.0 * d["nx"] * d["ny"] * d["nz"] * d["n_steps"]


class Result:
    def __init__(self, rid, F, grad, t_arrival, t_admit, t_done):
        self.id, self.F, self.grad = rid, F, grad
        self.t_arrival, self.t_admit, self.t_done = t_arrival, t_admit, t_done

    @property
    def latency(self):
        return self.t_done - self.t_arrival


def evaluate(req, stream=None):
    """One gradient evaluation on the current device (no server)."""
    p = Problem(req.desc, req.bg, req.m1, req.m2, req.gamma, stream=stream)
    try:
        p.set_density(req.rho)
        F, _ = p.forward()
        p.adjoint()
        g = p.gradient()
    finally:
        p.close()
    return F, g


class GradientServer:
    """submit(request) -> Future[Result].  max_slots requests on the device at once, their summed
    footprints within hbm_budget bytes."""

    def __init__(self, max_slots=8, hbm_budget=None, device=0):
        import torch
        self.torch = torch
        self.device = device
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget = int(0.8 * free)
        self.hbm_budget = hbm_budget
        self.max_slots = max_slots
        self.cv = threading.Condition()
        self.waiting = collections.deque()
        self.in_use = 0
        self.active = 0
        self.closed = False
        self.peak_active = 0
        self.peak_in_use = 0
        self.pool = cf.ThreadPoolExecutor(max_workers=max_slots)
        self.dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self.dispatcher.start()

    def submit(self, req):
        """Queue a request; an invalid or oversized one fails its own future, nothing else."""
        fut = cf.Future()
        try:
            fp = req.footprint()
        except Exception as e:
            fut.set_exception(e)
            return fut
        if fp > self.hbm_budget:
            fut.set_exception(N.FdtdError(2, f"request needs {fp} bytes, budget is {self.hbm_budget}"))
            return fut
        if req.t_arrival is None:
            req.t_arrival = time.perf_counter()
        with self.cv:
            self.waiting.append((req, fp, fut))
            self.cv.notify_all()
        return fut

    def _can_admit(self):
        return bool(self.waiting) and self.active < self.max_slots and \
            self.in_use + self.waiting[0][1] <= self.hbm_budget

    def _dispatch(self):
        while True:
            with self.cv:
                while not self._can_admit():
                    if self.closed and not self.waiting:
                        return
                    self.cv.wait()
                req, fp, fut = self.waiting.popleft()
                self.in_use += fp
                self.active += 1
                self.peak_active = max(self.peak_active, self.active)
                self.peak_in_use = max(self.peak_in_use, self.in_use)
            self.pool.submit(self._run, req, fp, fut, time.perf_counter())

    def _run(self, req, fp, fut, t_admit):
        torch = self.torch
        try:
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream(device=self.device)
            F, g = evaluate(req, stream=stream.cuda_stream)
            stream.synchronize()
            fut.set_result(Result(req.id, F, g, req.t_arrival, t_admit, time.perf_counter()))
        except Exception as e:  # the request fails, the server keeps serving
            fut.set_exception(e)
        finally:
            with self.cv:
                self.in_use -= fp
                self.active -= 1
                self.cv.notify_all()

    def close(self):
        """Serve everything already submitted, then stop."""
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        self.dispatcher.join()
        self.pool.shutdown(wait=True)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def replay_stream(requests, server=None, time_scale=1.0):
    """Submit requests at their (scaled) arrival times; return results in request order and the
    wall time from the first arrival to the last completion.  server=None runs them one after
    another in arrival order on the calling thread (the sequential baseline)."""
    t0 = time.perf_counter()
    futs, results = [], []
    for r in requests:
        due = t0 + r.t_arrival_rel * time_scale
        now = time.perf_counter()
        if due > now:
            time.sleep(due - now)
        r.t_arrival = due                       # latency counts from the stream's arrival time
        if server is None:
            start = time.perf_counter()
            F, g = evaluate(r)
            results.append(Result(r.id, F, g, due, start, time.perf_counter()))
        else:
            futs.append(server.submit(r))
    if server is not None:
        results = [f.result() for f in futs]
    wall = max(x.t_done for x in results) - t0
    return results, wall


def from_stream(items):
    """Requests from dicts with desc/bg/m1/m2/rho/gamma/id/t_arrival (the seeded serving stream)."""
    return [Request(it["desc"], it["bg"], it["m1"], it["m2"], it["rho"], it.get("gamma", 0.0), it.get("id"),
                    None, it["t_arrival"]) for it in items]


def latency_stats(results):
    lat = np.array([r.latency for r in results])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "n": int(lat.size)}
