"""Continuous-batching server for gradient evaluations (serving workload).

Requests of different grid sizes from concurrent optimisations arrive at any time.  The dispatcher
admits a waiting request (FIFO) as soon as a slot is free and its device footprint
(``fdtd_footprint_bytes``) fits the remaining HBM budget; every admitted request owns a handle whose
fields, CPML state, pole currents and DFTs stay resident on the device until its gradient is out.
Admitted requests go to one of two lanes:

* the batch lane (grids up to ``batch_max_cells``): the forward and adjoint runs of every request in
  the lane are advanced together by the persistent kernel (``fdtd_batch_run``: one captured CUDA graph
  per launch, work items from a device work queue, up to ``chunk_steps`` steps of every run per launch).
  Requests enter and leave between launches, so a request that arrives while others are on the GPU
  joins the next launch;
* the plain lane (larger grids, which fill the GPU on their own): each request runs its
  forward / adjoint / gradient as 16-step CUDA graphs on a stream of its own, next to the batch lane's
  launches.

Finished requests release their slot and memory immediately and the next waiting one is admitted.
Large grids (exclusive_cells) run one at a time: each nearly fills the HBM bandwidth alone, so two of
them side by side only slow each other, while smaller requests fill the SMs and the gaps between a large
grid's kernels; a request may overtake one that waits for a running large grid.  Measured on a GB300,
the persistent batch lane is slower than concurrent plain-lane requests at every grid size of the
serving stream (12-13 against 18-35 Gcell-updates/s on 48^3-96^3 grids), so the default routes every
request through the plain lane and the batch lane is an option (batch_max_cells).
Each result is bitwise independent of the mix: a request's state is private, every kernel is
deterministic, and a batched run's arithmetic does not depend on which runs share its launches.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time

import numpy as np

from . import _native as N
from .problem import Batch, Problem


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

    def cells(self):
        d = self.desc
        return d["nx"] * d["ny"] * d["nz"]

    def cell_updates(self):
        return 2.0 * self.cells() * self.desc["n_steps"]


class Result:
    def __init__(self, rid, F, grad, t_arrival, t_admit, t_done, lane=""):
        self.id, self.F, self.grad = rid, F, grad
        self.t_arrival, self.t_admit, self.t_done = t_arrival, t_admit, t_done
        self.lane = lane

    @property
    def latency(self):
        return self.t_done - self.t_arrival


def evaluate(req, stream=None):
    """One gradient evaluation on the current device, plain path (no server)."""
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
    """submit(request) -> Future[Result].

    max_slots requests on the device at once (at most 16 of them in the batch lane), their summed
    footprints within hbm_budget bytes.  batch_max_cells: grids with at most this many cells take the
    batch lane (0, the default: every request takes the plain lane; None: every FP32 request takes the
    batch lane).  chunk_steps: steps of every batched run per persistent launch; batch_blocks: blocks of
    those launches (0: as many as fit; fewer leave SMs to the plain lane's kernels).  plain_workers:
    plain-lane requests running at once.  exclusive_cells: grids with at least this many cells run one at
    a time (two of them side by side only share the HBM bandwidth each already nearly fills), and a
    waiting request may overtake one that waits for such a grid to finish (None: strict FIFO).

    The defaults are the measured best on the seeded 200-request stream on a GB300: the plain lane for
    every size, eight at a time, grids of 128^3 cells and more one at a time."""

    def __init__(self, max_slots=16, hbm_budget=None, device=0, batch_max_cells=0, chunk_steps=128,
                 plain_workers=8, batch_blocks=0, exclusive_cells=128 ** 3):
        import torch
        self.torch = torch
        self.device = device
        torch.cuda.set_device(device)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget = int(0.8 * free)
        self.hbm_budget = hbm_budget
        self.max_slots = max_slots
        self.batch_max_cells = batch_max_cells
        self.exclusive_cells = exclusive_cells
        self.exclusive_running = 0
        self.chunk_steps = chunk_steps
        self.cv = threading.Condition()
        self.waiting = collections.deque()
        self.in_use = 0
        self.active = 0
        self.closed = False
        self.peak_active = 0
        self.peak_in_use = 0
        self.peak_batched = 0
        self.batch_pending = 0
        self.launches = 0
        self.error = None
        self.stream = torch.cuda.Stream(device=device)
        self.batch_blocks = batch_blocks
        self.batch = self._new_batch()
        self.in_batch = {}          # Problem -> (request, future, footprint, t_admit, phase)
        self.plain_pool = cf.ThreadPoolExecutor(max_workers=plain_workers)
        self.dispatcher = threading.Thread(target=self._loop, daemon=True)
        self.dispatcher.start()

    # ---- public -------------------------------------------------------------------------------
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

    def close(self):
        """Serve everything already submitted, then stop."""
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        self.dispatcher.join()
        self.plain_pool.shutdown(wait=True)
        self.batch.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- dispatcher ---------------------------------------------------------------------------
    def _new_batch(self):
        b = Batch(self.stream.cuda_stream)
        if self.batch_blocks:
            b.set_blocks(self.batch_blocks)
        return b

    def _batch_lane(self, req):
        if req.desc.get("precision", 32) != 32:
            return False
        return self.batch_max_cells is None or req.cells() <= self.batch_max_cells

    def _exclusive(self, req):
        return self.exclusive_cells is not None and req.cells() >= self.exclusive_cells

    def _admissible(self, req, fp):
        if self.in_use + fp > self.hbm_budget:
            return False
        if self._exclusive(req) and self.exclusive_running > 0:
            return False
        return not self._batch_lane(req) or len(self.in_batch) + self.batch_pending < N.MAX_BATCH

    def _next_index(self):
        """Index of the request to admit next: the first waiting one, or, with exclusive_cells, the first
        one that is admissible when the head waits for a running large grid (large grids stay in FIFO
        order among themselves); None if none can start now."""
        if not self.waiting or self.active >= self.max_slots:
            return None
        for q, (req, fp, _) in enumerate(self.waiting):
            if self._admissible(req, fp):
                return q
            if self.exclusive_cells is None or not self._exclusive(req) or self.exclusive_running == 0:
                return None        # FIFO: only a head blocked by a running large grid lets others pass
        return None

    def _can_admit(self):
        return self._next_index() is not None

    def _release(self, fp, req=None):
        with self.cv:
            self.in_use -= fp
            self.active -= 1
            if req is not None and self._exclusive(req):
                self.exclusive_running -= 1
            self.cv.notify_all()

    def _admit_one(self):
        """Take the next admissible waiting request and start it in its lane (called with self.cv held)."""
        q = self._next_index()
        req, fp, fut = self.waiting[q]
        del self.waiting[q]
        self.in_use += fp
        self.active += 1
        if self._exclusive(req):
            self.exclusive_running += 1
        if self._batch_lane(req):
            self.batch_pending += 1             # in the batch lane from here on (counted before its submit)
        self.peak_active = max(self.peak_active, self.active)
        self.peak_in_use = max(self.peak_in_use, self.in_use)
        return req, fp, fut, time.perf_counter()

    def _start_batched(self, req, fp, fut, t_admit):
        with self.cv:
            self.batch_pending -= 1
        try:
            p = Problem(req.desc, req.bg, req.m1, req.m2, req.gamma, stream=self.stream.cuda_stream)
            try:
                p.set_density(req.rho)
                self.batch.submit(p)
            except Exception:
                p.close()
                raise
        except Exception as e:
            fut.set_exception(e)
            self._release(fp, req)
            return
        self.in_batch[p] = [req, fut, fp, t_admit, 0]
        self.peak_batched = max(self.peak_batched, len(self.in_batch))

    def _run_plain(self, req, fp, fut, t_admit):
        torch = self.torch
        try:
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream(device=self.device)
            F, g = evaluate(req, stream=stream.cuda_stream)
            stream.synchronize()
            fut.set_result(Result(req.id, F, g, req.t_arrival, t_admit, time.perf_counter(), "plain"))
        except Exception as e:  # the request fails, the server keeps serving
            fut.set_exception(e)
        finally:
            self._release(fp, req)

    def _finish_batched(self, p, status):
        req, fut, fp, t_admit, phase = self.in_batch[p]
        try:
            if status != 0:
                raise N.FdtdError(status, N.fdtd_last_error(p.h))
            if phase == 0:                      # forward run ended: its adjoint run joins the next launch
                self.batch.submit(p, adjoint=True)
                self.in_batch[p][4] = 1
                return
            F, _ = p.objective()
            g = p.gradient()
            fut.set_result(Result(req.id, F, g, req.t_arrival, t_admit, time.perf_counter(), "batch"))
        except Exception as e:
            fut.set_exception(e)
        del self.in_batch[p]
        p.close()
        self._release(fp, req)

    def _loop(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        while True:
            starts = []
            with self.cv:
                while True:
                    while self._can_admit():
                        starts.append(self._admit_one())
                    if starts or self.in_batch:
                        break
                    if self.closed and not self.waiting and self.active == 0:
                        return
                    self.cv.wait()
            for req, fp, fut, t_admit in starts:
                if self._batch_lane(req):
                    self._start_batched(req, fp, fut, t_admit)
                else:
                    self.plain_pool.submit(self._run_plain, req, fp, fut, t_admit)
            if not self.in_batch:
                continue
            try:
                done = self.batch.run(self.chunk_steps)
            except Exception as e:             # the batch is dead: fail its requests, start a new one
                self.error = e
                for p, (req, fut, fp, t_admit, phase) in list(self.in_batch.items()):
                    fut.set_exception(e)
                    p.close()
                    self._release(fp, req)
                self.in_batch.clear()
                self.batch.close()
                self.batch = self._new_batch()
                continue
            self.launches += 1
            for p, st in done:
                self._finish_batched(p, st)


def replay_stream(requests, server=None, time_scale=1.0):
    """Submit requests at their (scaled) arrival times; return results in request order and the
    wall time from the first arrival to the last completion.  server=None runs them one after
    another in arrival order on the calling thread (the sequential baseline, plain path)."""
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
            results.append(Result(r.id, F, g, due, start, time.perf_counter(), "sequential"))
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
