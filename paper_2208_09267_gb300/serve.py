"""Continuous-batching request loop for lattice solves.

Requests (one lattice each: size, volume fraction, relaxation time, a step
budget and optionally a steady-state residual target) arrive over time.  The
server keeps every admitted request's populations resident on the device in
its own lattice handle and advances all of them together: each macro-step is
one replay of a captured graph that runs K fused steps of every member
through the batched kernels of the library (lbm_vanse_batch_*).  Between
macro-steps it

  * admits arrived requests while the device-memory budget allows
    (admission by HBM budget, FIFO);
  * reads each member's check-step statistics (mass, residual, NaN flag);
  * retires members whose step budget is spent or whose residual reached the
    target: copies u and p to the host, records the latency (arrival to
    result on the host) and frees the member's memory, which lets waiting
    requests in.

Requests that arrive while others are on the GPU therefore join the running
batch at the next macro-step boundary: their work overlaps on the device with
the work of requests already running.  Per-cell arithmetic does not depend on
the batch, so a request's result is the same alone and in any mix.
"""
from __future__ import annotations

import math
import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import lbm
from .inputs import LatticeSpec


@dataclass
class Request:
    rid: int
    spec: LatticeSpec
    arrival: float                # seconds after the start of the run
    eps: np.ndarray | None = None  # phi field (host), generated by the client
    admitted: float | None = None
    finished: float | None = None
    steps_done: int = 0
    status: str = "queued"        # queued, running, done, converged, unstable, rejected
    residual: float = -1.0
    result: dict | None = None
    lattice: object = None
    bytes: int = 0

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


def request_bytes(spec: LatticeSpec, storage: str) -> int:
    nz, ny, nx = spec.shape
    base = lbm.device_bytes(spec.lattice, (nx, ny, nz), storage)
    return base + 3 * lbm.stored_cells(nx, ny, nz) * 4  # the residual buffer of a batch member


@dataclass
class ServerStats:
    completed: int = 0
    rejected: int = 0
    cell_updates: float = 0.0
    elapsed: float = 0.0
    latencies: list = field(default_factory=list)
    macro_steps: int = 0
    peak_members: int = 0
    peak_bytes: int = 0
    incomplete: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.array([np.nan])
        return {"completed": self.completed, "rejected": self.rejected,
                "solves_per_s": self.completed / self.elapsed if self.elapsed > 0 else 0.0,
                "glups": self.cell_updates / self.elapsed / 1e9 if self.elapsed > 0 else 0.0,
                "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)),
                "mean_latency_s": float(np.mean(lat)),
                "elapsed_s": self.elapsed, "macro_steps": self.macro_steps,
                "peak_members": self.peak_members, "peak_bytes": self.peak_bytes,
                "incomplete": self.incomplete}


class Server:
    """Continuous batching server on one GPU.

    storage: "fp16" (shifted half storage) or "fp32"; hbm_budget: bytes of
    device memory the admitted requests may hold together; macro_steps: K,
    steps per graph replay (even); keep_results: copy u and p of every
    finished request to the host."""

    def __init__(self, storage="fp16", hbm_budget=80e9, macro_steps=100, max_members=1024,
                 max_tiles=1 << 20, tile_cells=None, stream=None, keep_results=True,
                 fp16_scale_log2=10):
        if macro_steps < 2 or macro_steps % 2:
            raise ValueError("macro_steps must be even and >= 2")
        self.storage = storage
        self.budget = int(hbm_budget)
        self.K = int(macro_steps)
        self.stream = stream
        self.keep_results = keep_results
        self.fp16_k = fp16_scale_log2
        self.batch = lbm.Batch(max_members=max_members, max_tiles=max_tiles,
                               tile_cells=tile_cells, stream=stream, storage=storage)
        self.queue = deque()
        self.active: list[Request] = []
        self.done: list[Request] = []
        self.used = 0
        self.lock = threading.Lock()
        self.stats = ServerStats()

    # -- client side ---------------------------------------------------------
    def submit(self, req: Request):
        with self.lock:
            self.queue.append(req)

    # -- server side ---------------------------------------------------------
    def _admit(self, now: float):
        with self.lock:
            while self.queue and self.queue[0].arrival <= now:
                req = self.queue[0]
                need = request_bytes(req.spec, self.storage)
                if need > self.budget:
                    self.queue.popleft()
                    req.status = "rejected"
                    self.stats.rejected += 1
                    self.done.append(req)
                    continue
                if self.used + need > self.budget:
                    break   # FIFO: wait until memory frees up
                self.queue.popleft()
                self._start(req, need, now)

    def _start(self, req: Request, need: int, now: float):
        s = req.spec
        nz, ny, nx = s.shape
        lat = lbm.Lattice(s.lattice, (nx, ny, nz), tau=s.tau, storage=self.storage,
                          stream=self.stream, fp16_scale_log2=self.fp16_k)
        eps = req.eps if req.eps is not None else s.eps()
        lat.set_epsilon(np.asarray(eps, np.float32).ravel())
        lat.set_force(s.g)
        lat.init_equilibrium()
        self.batch.add(lat, s.steps)
        req.lattice = lat
        req.bytes = need
        req.admitted = now
        req.status = "running"
        self.used += need
        self.active.append(req)
        self.stats.peak_members = max(self.stats.peak_members, len(self.active))
        self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)

    def _retire(self, req: Request, now_fn, status: str):
        lat = req.lattice
        if self.keep_results:
            # the read-back through the library's fixed staging array takes no
            # device memory outside the admission budget (the server loop is
            # single-threaded, so its calls never overlap)
            if lat.n <= lbm.NOALLOC_MAX_CELLS:
                m = lat.moments_noalloc()
            else:
                m = lat.moments(f64=False)
            req.result = {"u": m["u"], "p": m["p"]}
        req.finished = now_fn()
        req.status = status
        self.batch.remove(lat)
        lat.close()
        req.lattice = None
        self.used -= req.bytes
        self.stats.completed += 1
        self.stats.latencies.append(req.latency)
        self.stats.cell_updates += req.spec.cells * req.steps_done
        self.done.append(req)

    def step(self, now_fn):
        """One macro-step of every active request; retire the finished."""
        if not self.active:
            return
        self.batch.step(self.K, check=True)
        self.stats.macro_steps += 1
        finished = []
        for req in self.active:
            st = self.batch.stats(req.lattice)
            req.steps_done = st["steps_done"]
            req.residual = st["residual"]
            if st["nan_seen"]:
                finished.append((req, "unstable"))
            elif req.steps_done >= req.spec.steps:
                finished.append((req, "done"))
            elif (req.spec.residual_tol > 0 and 0 <= req.residual <= req.spec.residual_tol):
                finished.append((req, "converged"))
        for req, status in finished:
            self.active.remove(req)
            self._retire(req, now_fn, status)

    def run(self, requests, timeout_s: float = 3600.0):
        """(see below); requests still queued or running when timeout_s
        passes are counted as incomplete."""
        """Serve a list of requests whose .arrival are seconds after the start
        (arrivals are simulated against the wall clock); returns the stats
        summary."""
        for r in sorted(requests, key=lambda r: r.arrival):
            self.submit(r)
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0
        while True:
            t = now()
            if t > timeout_s:
                break
            self._admit(t)
            if self.active:
                self.step(now)
                continue
            with self.lock:
                if not self.queue:
                    break
                wait = self.queue[0].arrival - now()
            if wait > 0:
                time.sleep(min(wait, 0.05))
        self.stats.elapsed = now()
        self.stats.incomplete = len(self.active) + len(self.queue)
        return self.stats.summary()

    def close(self):
        for req in list(self.active):
            self.batch.remove(req.lattice)
            req.lattice.close()
        self.active.clear()
        self.batch.close()


def run_sequential(requests, storage="fp32", check_every=100, stream=None, keep_results=True,
                   timeout_s: float = float("inf")):
    """The plain per-request baseline: one solver per request, first come
    first served, each run to its step budget or residual target alone.
    Requests not started by timeout_s are left queued."""
    stats = ServerStats()
    t0 = time.perf_counter()

    def now():
        return time.perf_counter() - t0
    for req in sorted(requests, key=lambda r: r.arrival):
        if now() > timeout_s:
            break
        wait = req.arrival - now()
        if wait > 0:
            time.sleep(wait)
        s = req.spec
        nz, ny, nx = s.shape
        lat = lbm.Lattice(s.lattice, (nx, ny, nz), tau=s.tau, storage=storage, stream=stream)
        eps = req.eps if req.eps is not None else s.eps()
        lat.set_epsilon(np.asarray(eps, np.float32).ravel())
        lat.set_force(s.g)
        lat.init_equilibrium()
        st = lat.step(s.steps, residual_tol=s.residual_tol, check_every=check_every)
        req.steps_done = st["steps_done"]
        req.residual = st["residual"]
        if keep_results:
            m = lat.moments(f64=False)
            req.result = {"u": m["u"], "p": m["p"]}
        req.finished = now()
        req.status = "converged" if st["converged"] else "done"
        lat.close()
        stats.completed += 1
        stats.latencies.append(req.latency)
        stats.cell_updates += s.cells * req.steps_done
    stats.elapsed = now()
    stats.incomplete = len(requests) - stats.completed
    return stats.summary()


def make_requests(rate: float, count: int, seed_offset: int = 5000, sides=(32, 192),
                  steps=(500, 20000), residual_share=0.5, sphere_share=0.5, with_eps=True):
    """Poisson request trace with client-generated phi fields."""
    from .inputs import poisson_requests
    from .inputs import cached_eps
    out = []
    for j, (t, spec) in enumerate(poisson_requests(rate, count, seed_offset, sides, steps,
                                                   residual_share, sphere_share)):
        out.append(Request(j, spec, t, cached_eps(spec) if with_eps else None))
    return out
