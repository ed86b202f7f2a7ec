"""Throughput of the fused VANSE lattice Boltzmann step on GB300.

Workload (default): D3Q19, 256^3 periodic, FP32 storage, tau = 0.6, body
force 1e-6 x, space-time varying volume fraction
phi = 0.7 + 0.2 sin(2 pi x/L) cos(2 pi y/L) sin(2 pi z/L + 2 pi t/T), T = 1000
steps, refreshed (phi_ref, d_t phi) every 10 steps, with a check step (FP64
mass/momentum sums and the velocity residual) every 100 steps.  One bench
step = one fused time step of the whole lattice.  The populations (1.27 GB in FP32) are
far larger than L2 (129 MB), so no flush is needed between steps.

Output: one JSON line (rank 0).  ``value`` = GLUPS (10^9 cell updates per
second) with inputs resident in HBM; ``e2e`` = the same through the C ABI
with host buffers (phi refreshes uploaded from pinned host memory, the
check-step statistics read back); ``roofline`` = the step kernel's
algorithmic bytes per launch over its average CUDA-event duration, against
the measured HBM copy bandwidth.  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_DEFAULT = 256
T_PERIOD = 1000.0
K_EPS = 10
K_CHECK = 100  # a check step (FP64 sums, velocity residual) every 100 steps
TAU = 0.6
G = (1e-6, 0.0, 0.0)
Q = 19
def metric_name(L: int = 256) -> str:
    return f"GLUPS (D3Q19 VANSE step, {L}^3, FP32)"


def bytes_per_cell(storage: str) -> int:
    """Algorithmic bytes per cell update: one read and one write of each
    population (AA pattern) plus phi_ref and d_t phi, 4 B each."""
    b = {"fp32": 4, "fp16": 2}[storage]
    return 2 * Q * b + 4 + 4


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(storage: str, kernel_src_hash: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    source has not changed since it was captured."""
    path = os.path.join(ROOT, "profiles", f"step_row_d3q19_{storage}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != kernel_src_hash:
        return None
    return float(t.group(1))


def kernel_source_hash() -> str:
    """Hash of the D3Q19 row kernel's sources with comments and blank space
    removed: a profile stays valid across comment edits, not code edits."""
    h = hashlib.sha256()
    for name in ("step_row.cuh", "step_row_pair.cuh", "step_fast.cuh", "step_fast_d3q19.cu", "lattice.cuh",
                 "internal.h"):
        with open(os.path.join(ROOT, "paper_2208_09267_gb300", "csrc", name)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


class ClockSampler:
    """SM clock and clock-event reasons sampled DURING a timed region.

    Reads NVML directly (libnvidia-ml through ctypes, every 2 ms, so that a
    timed region of a few milliseconds still gets samples); falls back to
    ``nvidia-smi -lms 20`` where NVML cannot be loaded.  Reads only: it
    changes no setting of the GPU."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    SMI_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_s: float = 0.002):
        self.gpu = gpu_index
        self.interval = interval_s
        self.samples = []      # (sm_mhz, max_mhz, reason names)
        self.proc = None
        self.thread = None
        self.stop = threading.Event()
        self.source = None

    def _nvml(self):
        import ctypes
        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                lib = ctypes.CDLL(name)
                break
            except OSError:
                lib = None
        if lib is None or lib.nvmlInit_v2() != 0:
            return None
        dev = ctypes.c_void_p()
        handle = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.gpu).uuid)
            key = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            if lib.nvmlDeviceGetHandleByUUID(key.encode(), ctypes.byref(dev)) == 0:
                handle = dev
        except Exception:
            handle = None
        if handle is None:
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu), ctypes.byref(dev)) != 0:
                return None
            handle = dev
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        return lib, handle, reasons_fn

    def _poll_nvml(self, lib, handle, reasons_fn):
        import ctypes
        clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(handle, 1, ctypes.byref(clk)) == 0
                    and lib.nvmlDeviceGetMaxClockInfo(handle, 1, ctypes.byref(mx)) == 0
                    and reasons_fn(handle, ctypes.byref(rs)) == 0):
                names = [v for k, v in self.REASONS.items() if rs.value & k]
                self.samples.append((float(clk.value), float(mx.value), names))
            self.stop.wait(self.interval)

    def _read_smi(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9 and p[1].replace(".", "").isdigit() and p[2].replace(".", "").isdigit():
                self.samples.append((float(p[1]), float(p[2]),
                                     [names[j] for j in range(4) if p[5 + j].lower() == "active"]))

    def __enter__(self):
        nv = None
        try:
            nv = self._nvml()
        except Exception:
            nv = None
        if nv is not None:
            self.source = "nvml"
            self.thread = threading.Thread(target=self._poll_nvml, args=nv, daemon=True)
            self.thread.start()
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.SMI_Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi"
            self.thread = threading.Thread(target=self._read_smi, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [s[0] for s in self.samples]
        mx = [s[1] for s in self.samples]
        reasons = sorted({r for s in self.samples for r in s[2]})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": reasons,
                "samples": len(self.samples), "source": self.source}


def eps_fields(L, t):
    from paper_2208_09267_gb300 import inputs
    e, d = inputs.eps_travelling_wave(L, float(t), T=T_PERIOD)
    return e.ravel().astype(np.float32), d.ravel().astype(np.float32)


def max_over_ranks(value: float, device) -> float:
    """The largest value over the ranks of the process group (the job's
    time is its slowest rank's); the value itself with one rank."""
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def aggregate_glups(cells_per_rank: int, steps: int, max_ms: float, world: int) -> float:
    """Whole-job throughput: every rank advances its own replica of
    cells_per_rank cells by `steps` steps; the job takes the slowest rank's
    time (weak scaling, no data-path collective)."""
    return cells_per_rank * world * steps / (max_ms * 1e-3) / 1e9


def run_gpu(args, rank, world):
    import torch

    from paper_2208_09267_gb300 import lbm

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    L = args.size
    N = L ** 3
    total_steps = args.warmup + args.steps
    nref = (total_steps + K_EPS - 1) // K_EPS + 1

    # phi_ref / d_t phi at every refresh, resident on the device and pinned on the host
    host_e = torch.empty((nref, N), dtype=torch.float32, pin_memory=True)
    host_d = torch.empty((nref, N), dtype=torch.float32, pin_memory=True)
    for j in range(nref):
        e, d = eps_fields(L, j * K_EPS)
        host_e[j].numpy()[:] = e
        host_d[j].numpy()[:] = d
    dev_e = host_e.to(f"cuda:{dev}")
    dev_d = host_d.to(f"cuda:{dev}")

    def make(storage):
        lat = lbm.Lattice("D3Q19", (L, L, L), tau=TAU, storage=storage,
                          stream=stream.cuda_stream, block=tuple(args.block))
        lat.set_epsilon(dev_e[0], dev_d[0], 0)
        lat.set_force(G)
        lat.init_equilibrium()
        return lat

    def device_run(lat, steps, timed):
        """steps fused steps with refreshes from device memory; returns
        (total_ms, kernel_ms, kernels) when timed."""
        ev = []
        n = lat.steps_done
        done = 0
        while done < steps:
            k = min(K_EPS - (n % K_EPS), steps - done)
            # plain steps, and a check step where the chunk ends on a multiple of K_CHECK
            ce = 0 if (n + k) % K_CHECK == 0 else -1
            if timed:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                lat.step(k, check_every=ce)
                b.record(stream)
                ev.append((a, b, k))
            else:
                lat.step(k, check_every=ce)
            n += k
            done += k
            if n % K_EPS == 0:
                j = n // K_EPS
                lat.set_epsilon(dev_e[j], dev_d[j], n)
        return ev

    results = {}
    tuning = {}
    if args.tune:
        # a bounded sweep of the row kernel's launch shapes on this lattice
        # (cached per size bucket; the lattices below read the cache)
        from paper_2208_09267_gb300 import tune
        for storage in args.storages:
            best, ms = tune.tune_step("D3Q19", storage, (L, L, L), tau=TAU, steps=10, warmup=3,
                                      blocks=[(256, 1)])
            tuning[storage] = {"best": best, "ms_per_step": ms}
    for storage in args.storages:
        lat = make(storage)
        device_run(lat, args.warmup, False)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        c0 = lbm.launch_count()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev) as clk:
            t0.record(stream)
            ev = device_run(lat, args.steps, True)
            t1.record(stream)
            torch.cuda.synchronize()
        launches = lbm.launch_count() - c0
        total_ms = t0.elapsed_time(t1)
        step_ms = sum(a.elapsed_time(b) for a, b, _ in ev)
        nk = sum(k for _, _, k in ev)
        if world > 1:
            total_ms = max_over_ranks(total_ms, f"cuda:{dev}")
        st = lat.step(1)  # one check step (not timed) to confirm the run is sane
        if st["nan_seen"]:
            raise RuntimeError(f"{storage}: NaN after the timed steps")
        kname = "step_row_kernel" if lat.row_kernel else "step_fast_kernel"
        results[storage] = {"total_ms": total_ms, "kernel_ms": step_ms / nk, "launches": launches,
                            "clocks": clk.summary(), "mass": st["mass"],
                            "kernel": f"{kname}<D3Q19,{'float' if storage == 'fp32' else '__half'}>",
                            "launch_shape": lat.launch_shape, "tuned_from": lat.tuned_from}
        lat.close()

    # end to end through the C ABI with host buffers (FP32).  The refreshes
    # reach the library the way a streaming application would hand them
    # over: a producer (twelve host threads) copies each refresh's phi_ref and
    # d_t phi into a ring of six pinned buffers, ahead of use.  The main
    # loop stages the next refresh (H2D copy and checks on the library's copy
    # stream), steps, and commits it, so the upload overlaps the steps.  A
    # fresh pinned buffer per refresh would instead pay the host-memory
    # first-touch of the device's DMA (measured ~8 GB/s against ~170 GB/s
    # once warm).
    e2e = None
    if not args.no_e2e:
        import queue
        ring = 6
        st_e = torch.empty((ring, N), dtype=torch.float32, pin_memory=True)
        st_d = torch.empty((ring, N), dtype=torch.float32, pin_memory=True)
        st_e_np = [st_e[i].numpy() for i in range(ring)]
        st_d_np = [st_d[i].numpy() for i in range(ring)]
        free = threading.Semaphore(ring)
        ready = queue.Queue()

        import concurrent.futures as cf
        nthr = 12
        pool = cf.ThreadPoolExecutor(max_workers=nthr)
        parts = [(i * N // nthr, (i + 1) * N // nthr) for i in range(nthr)]

        def producer(first, count):
            for q in range(count):
                free.acquire()
                slot = (first + q) % ring
                src_e, src_d = host_e[first + q].numpy(), host_d[first + q].numpy()

                def fill(ab, slot=slot, src_e=src_e, src_d=src_d):
                    a, b = ab
                    np.copyto(st_e_np[slot][a:b], src_e[a:b])
                    np.copyto(st_d_np[slot][a:b], src_d[a:b])
                list(pool.map(fill, parts))   # the host threads fill the slot
                ready.put(slot)

        lat = lbm.Lattice("D3Q19", (L, L, L), tau=TAU, storage=args.storages[0],
                          stream=stream.cuda_stream, block=tuple(args.block))
        lat.set_force(G)
        nwarm = args.warmup // K_EPS
        chunks = max(1, args.steps // K_EPS)
        prod = threading.Thread(target=producer, args=(0, min(nref, nwarm + chunks + 1)), daemon=True)
        prod.start()
        slot = ready.get()
        lat.set_epsilon(st_e_np[slot], st_d_np[slot], 0)
        free.release()
        lat.init_equilibrium()
        def chunk(n_next):
            slot = ready.get()
            lat.stage_epsilon(st_e_np[slot], st_d_np[slot], n_next)  # H2D (pinned) on the copy stream
            lat.step(K_EPS)                                          # ends with a check step: stats D2H
            lat.commit_epsilon()
            free.release()                                           # the slot may be refilled now
        for j in range(nwarm):
            chunk((j + 1) * K_EPS)
        torch.cuda.synchronize()
        n0 = lat.steps_done
        t = time.perf_counter()
        for j in range(chunks):
            chunk(n0 + (j + 1) * K_EPS)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        prod.join()
        pool.shutdown()
        e2e = {"value": N * chunks * K_EPS / dt / 1e9, "unit": "GLUPS",
               "h2d_bytes_per_step": 2 * 4 * N / K_EPS,
               "d2h_bytes_per_step": 120 / K_EPS,
               "note": "phi_ref and d_t phi of every refresh (each 10 steps) copied from a ring of "
                       "pinned host buffers filled by host threads, staged on the library's copy "
                       "stream during the 10 steps before it and committed after them; each "
                       "10-step call reads its check statistics back"}
        lat.close()
    return results, e2e, tuning


def run_porous(steps=200, warmup=10, shape=(512, 256, 256), storages=("fp32", "fp16")):
    """The porous channel: D3Q27, 512x256x256, random spheres (radius 4-12,
    packing 0.35) smoothed by a Gaussian (sigma 3) to phi in [0.4, 1], walls
    at y = 0 and 255, periodic x and z, tau 0.6, body force 1e-6 x, static
    phi.  GLUPS and the fraction of the copy bandwidth at 2 Q b + 4 bytes
    per cell (220 FP32, 112 FP16), timed with CUDA events over plain steps."""
    import torch

    from paper_2208_09267_gb300 import inputs, lbm
    nx, ny, nz = shape
    t0 = time.perf_counter()
    eps = inputs.eps_random_spheres((nz, ny, nx), seed_offset=2, wall_axis=1).ravel().astype(np.float32)
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    peak, _ = peak_hbm()
    out = {"workload": f"D3Q27 porous channel {nx}x{ny}x{nz}, walls y, static phi (spheres r 4-12, "
                       f"packing 0.35, Gaussian sigma 3), tau 0.6, g 1e-6 x", "steps": steps,
           "phi_generation_s": gen_s}
    for storage in storages:
        lat = lbm.Lattice("D3Q27", shape, tau=0.6, storage=storage, walls=2, stream=stream.cuda_stream)
        lat.set_epsilon(eps)
        lat.set_force(G)
        lat.init_equilibrium()
        lat.step(warmup, check_every=-1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            a.record(stream)
            lat.step(steps, check_every=-1)
            b.record(stream)
            torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        st = lat.step(1)
        bpc = 2 * 27 * (4 if storage == "fp32" else 2) + 4
        cells = nx * ny * nz
        out[storage] = {"glups": cells / (ms * 1e-3) / 1e9, "ms_per_step": ms, "bytes_per_cell": bpc,
                        "achieved_gbs": bpc * cells / (ms * 1e-3) / 1e9,
                        "frac": bpc * cells / (ms * 1e-3) / 1e9 / peak,
                        "kernel": "step_row_kernel" if lat.row_kernel else "step_fast_kernel",
                        "nan_seen": bool(st["nan_seen"]), "clocks": clk.summary()}
        lat.close()
    return out


def batch_bytes(specs, storage):
    """Algorithmic bytes of one step of every lattice of a batch: per cell one
    read and one write of each population plus phi_ref (static phi)."""
    b = {"fp32": 4, "fp16": 2}[storage]
    q = {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}
    return sum(s.cells * (2 * q[s.lattice] * b + 4) for s in specs)


def run_batched(count=256, steps=1000, storages=("fp16", "fp32")):
    """The batched workload: 256 independent lattices (half D2Q9 squares of
    side 32..512, half D3Q19 cubes of side 32..128, product-sine phi, tau in
    [0.55, 1.2]), 1000 steps each, advanced together by the batched
    graph-captured kernels, against the plain per-lattice FP32 path (one
    handle per lattice, stepped one after the other).  Returns GLUPS,
    lattices solved per second and, for the batched legs, the aggregate
    fraction of the copy bandwidth (algorithmic bytes of every member)."""
    import torch

    from paper_2208_09267_gb300 import inputs, lbm
    specs = inputs.batch_specs(count=count, steps=steps)
    cells = sum(s.cells for s in specs)
    stream = torch.cuda.current_stream().cuda_stream
    peak, peak_kind = peak_hbm()
    out = {"lattices": count, "steps": steps, "cells": cells}

    def make(storage, s):
        nz, ny, nx = s.shape
        lat = lbm.Lattice(s.lattice, (nx, ny, nz), tau=s.tau, storage=storage, stream=stream)
        lat.set_epsilon(eps_of[id(s)])
        lat.set_force(s.g)
        lat.init_equilibrium()
        return lat
    eps_of = {id(s): s.eps().ravel().astype(np.float32) for s in specs}
    for storage in storages:
        lats = [make(storage, s) for s in specs]
        b = lbm.Batch(max_members=count, max_tiles=sum((lt.stored + 4095) // 4096 for lt in lats) + 8,
                      stream=stream, storage=storage)
        # replays of k steps (their graph is captured in the warm-up replay)
        k = 100 if steps % 100 == 0 else (50 if steps % 50 == 0 else 10)
        for lt in lats:
            b.add(lt, steps + k)
        b.step(k)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(steps // k):
            b.step(k)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        b.close()
        for lt in lats:
            lt.close()
        gbs = batch_bytes(specs, storage) * steps / dt / 1e9
        out[f"batched_{storage}"] = {"glups": cells * steps / dt / 1e9, "solves_per_s": count / dt,
                                     "seconds": dt, "achieved_gbs": gbs, "frac": gbs / peak,
                                     "peak_kind": f"{peak_kind} copy bandwidth",
                                     "tile_cells_tuned_from": b.tuned_from}
    # plain per-lattice FP32: one solver per lattice, each stepped alone
    lats = [make("fp32", s) for s in specs]
    for lt in lats:
        lt.step(70)  # captures the lattice's 64-step graph outside the timed region
    torch.cuda.synchronize()
    t = time.perf_counter()
    for lt in lats:
        lt.step(steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    for lt in lats:
        lt.close()
    gbs = batch_bytes(specs, "fp32") * steps / dt / 1e9
    out["per_lattice_fp32"] = {"glups": cells * steps / dt / 1e9, "solves_per_s": count / dt,
                               "seconds": dt, "achieved_gbs": gbs, "frac": gbs / peak}
    return out


def _fifo(arrivals, durations):
    """Latencies and makespan of one sequential server (first come, first
    served) for requests arriving at `arrivals` that take `durations`."""
    t, lat = 0.0, []
    for a, d in sorted(zip(arrivals, durations)):
        t = max(t, a) + d
        lat.append(t - a)
    return lat, t


def run_serving(rates=(10.0, 20.0, 50.0, 100.0, 200.0, 500.0), window_s=4.0, max_requests=16,
                sides=(32, 192), steps=(500, 20000), serve_timeout_s=30.0, seq_timeout_s=90.0):
    """The served workload: for each arrival rate, a Poisson stream of D3Q19
    solves (side log-uniform in `sides`, random-sphere or sine phi 50/50, a
    step budget log-uniform in `steps`, half of them with a steady-state
    residual target of 1e-8 capped by that budget), admitted by an 80 GB HBM
    budget and served with continuous batching in FP16-shifted storage,
    against plain per-request FP32 (one solver per request, sequential).

    Bounded trace: the requests arriving within `window_s` seconds, at most
    `max_requests` (the same problems at every rate), the served run cut at
    `serve_timeout_s`; the line states how many completed.  The sequential
    FP32 server solves each problem once (its compute time per request does
    not depend on the rate); its latencies at each rate follow from the
    arrival times by first-come-first-served queueing of those measured
    durations.  Reports solves/s and p50/p99 latency (arrival to result on
    the host) per rate, and the relative L2 distance of the FP16 velocity to
    FP32 run to the same step count: for budget-limited requests the
    sequential run itself, for requests the server retired on the residual
    target an FP32 run of exactly the steps the FP16 request took."""
    import dataclasses

    import torch

    from paper_2208_09267_gb300 import serve
    stream = torch.cuda.current_stream().cuda_stream
    count = int(min(max_requests, max(4, max(rates) * window_s)))
    out = {"trace": f"Poisson arrivals, D3Q19 side log-uniform {sides}, steps log-uniform {steps}, "
                    f"half with residual 1e-8, spheres or sine phi 50/50, 80 GB budget, {count} requests "
                    f"per rate (the same problems at every rate), served run cut at {serve_timeout_s:g} s",
           "rates": {}}
    # sequential FP32: every problem once, back to back
    seq_reqs = [serve.Request(r.rid, r.spec, 0.0, r.eps)
                for r in serve.make_requests(rates[0], count, sides=sides, steps=steps, seed_offset=5000)]
    t_prev = 0.0
    seq = serve.run_sequential(seq_reqs, storage="fp32", check_every=100, stream=stream,
                               timeout_s=seq_timeout_s)
    durations = {}
    for r in sorted(seq_reqs, key=lambda r: r.rid):
        if r.finished is not None:
            durations[r.rid] = r.finished - t_prev
            t_prev = r.finished
    out["sequential_fp32_solve"] = {"completed": seq["completed"], "seconds": seq["elapsed_s"],
                                    "glups": seq["glups"]}
    first_served = None
    for rate in rates:
        reqs = serve.make_requests(rate, count, sides=sides, steps=steps, seed_offset=5000)
        srv = serve.Server(storage="fp16", hbm_budget=80e9, macro_steps=100, stream=stream,
                           keep_results=True)
        served = srv.run(reqs, timeout_s=serve_timeout_s)
        srv.close()
        if first_served is None:
            first_served = reqs
        done = [r for r in reqs if r.rid in durations]
        lat, makespan = _fifo([r.arrival for r in done], [durations[r.rid] for r in done])
        seq_rate = {"completed": len(done), "solves_per_s": len(done) / makespan if makespan > 0 else 0.0,
                    "p50_latency_s": float(np.percentile(lat, 50)) if lat else None,
                    "p99_latency_s": float(np.percentile(lat, 99)) if lat else None}
        out["rates"][f"{rate:g}"] = {"requests": count, "served_fp16": served, "sequential_fp32": seq_rate}
    # FP16 against FP32 at the same step count
    errs = {"budget": [], "residual": []}
    seq_by_id = {r.rid: r for r in seq_reqs}
    for a in first_served:
        if a.result is None:
            continue
        b = seq_by_id.get(a.rid)
        if a.status == "converged":
            spec = dataclasses.replace(a.spec, steps=a.steps_done, residual_tol=0.0)
            ref = [serve.Request(a.rid, spec, 0.0, a.eps)]
            serve.run_sequential(ref, storage="fp32", check_every=100, stream=stream)
            b, kind = ref[0], "residual"
        else:
            kind = "budget"
        if b is None or b.result is None or b.steps_done != a.steps_done:
            continue
        ua, ub = a.result["u"].astype(np.float64), b.result["u"].astype(np.float64)
        nb = np.linalg.norm(ub)
        if nb > 0:
            errs[kind].append(float(np.linalg.norm(ua - ub) / nb))
    out["fp16_vs_fp32_u_rel_l2"] = {k: {"max": max(v) if v else None, "compared": len(v)} for k, v in errs.items()}
    return out


def _oracle_rate(P, f, steps, threads):
    """GLUPS of `steps` oracle steps on `threads` host threads (0 = all)."""
    import oracle
    oracle.set_threads(threads)
    t = time.perf_counter()
    P.run(f, 0, steps)
    dt = time.perf_counter() - t
    return P.n * steps / dt / 1e9, dt


def cpu_baseline(sample_L=48, steps=None, budget_s=15.0, plan=True):
    """The FP64 oracle on the host cores, timed on a bounded sample of the
    same workload (a sample_L^3 lattice with the same phi recipe, all cores),
    and with `plan`, bounded samples of the other workloads: the 64^2 D2Q9
    case run in full on one thread, the D3Q19 sample on one thread, the
    D3Q19 workload at 64^3 and 128^3, a D3Q27 porous-channel block (64 x 32
    x 32, walls on y) and eight lattices of the batched workload (a few steps
    each), all cores."""
    import oracle
    from paper_2208_09267_gb300 import inputs
    oracle.build()
    cores = os.cpu_count() or 1
    e, d = eps_fields(sample_L, 0)
    P = oracle.Problem("D3Q19", sample_L, sample_L, sample_L, tau=TAU, eps_ref=e, deps_dt=d, g=G)
    f = P.init()
    oracle.set_threads(0)
    t = time.perf_counter()
    f = P.run(f, 0, 2)
    per = (time.perf_counter() - t) / 2
    if steps is None:
        steps = max(2, int(budget_s / max(per, 1e-6)))
    value, dt = _oracle_rate(P, f, steps, 0)
    out = {"value": value, "unit": "GLUPS", "cores": cores, "kind": "oracle",
           "sample": f"D3Q19 {sample_L}^3 lattice, same phi recipe and tau, {steps} steps, "
                     f"FP64 oracle with {cores} OpenMP threads ({dt:.1f} s)"}
    if not plan:
        return out
    legs = {}
    # the 64^2 D2Q9 FP64 case, all 1000 steps, one thread
    e1 = inputs.eps_static_sine(64)
    P1 = oracle.Problem("D2Q9", 64, 64, 1, tau=0.8, eps_ref=e1, g=(1e-6, 0, 0))
    legs["d2q9_64x64_1000_steps_1_thread"] = _oracle_rate(P1, P1.init(), 1000, 1)[0]
    # the space-time varying D3Q19 sample on one thread, 10 steps
    legs[f"d3q19_{sample_L}^3_1_thread"] = _oracle_rate(P, f, 10, 1)[0]
    # the travelling-wave workload at 64^3 and 128^3 (the coarse levels of
    # its refinement study), a few steps each, all cores
    for Ls, ks in ((64, 10), (128, 3)):
        e2, d2 = eps_fields(Ls, 0)
        P2 = oracle.Problem("D3Q19", Ls, Ls, Ls, tau=TAU, eps_ref=e2, deps_dt=d2, g=G)
        legs[f"d3q19_{Ls}^3_all_cores"] = _oracle_rate(P2, P2.init(), ks, 0)[0]
    # a block of the porous channel: D3Q27, walls on y, static phi
    shape = (32, 32, 64)
    e3 = inputs.eps_random_spheres(shape, seed_offset=2, wall_axis=1)
    P3 = oracle.Problem("D3Q27", 64, 32, 32, tau=0.6, walls=2, eps_ref=e3, g=G)
    legs["d3q27_porous_64x32x32_all_cores"] = _oracle_rate(P3, P3.init(), 20, 0)[0]
    # eight lattices of the batched workload, 5 steps each, all cores
    specs = inputs.batch_specs(count=256)[::32]
    cells, secs = 0, 0.0
    for sp in specs:
        nz, ny, nx = sp.shape
        Pb = oracle.Problem(sp.lattice, nx, ny, nz, tau=sp.tau, eps_ref=sp.eps(), g=sp.g)
        _, dtb = _oracle_rate(Pb, Pb.init(), 5, 0)
        cells += sp.cells * 5
        secs += dtb
    legs["batched_8_lattices_all_cores"] = cells / secs / 1e9
    out["plan_glups"] = legs
    oracle.set_threads(0)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--size", type=int, default=L_DEFAULT)
    ap.add_argument("--block", type=int, nargs=2, default=[0, 0])
    ap.add_argument("--storages", nargs="+", default=["fp32", "fp16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the launch-shape sweep before the timed legs")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-porous", action="store_true")
    ap.add_argument("--porous-steps", type=int, default=200)
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[10.0, 20.0, 50.0, 100.0, 200.0, 500.0])
    ap.add_argument("--serve-window", type=float, default=4.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    L = args.size
    N = L ** 3
    config = {"workload": f"D3Q19 VANSE BGK {L}^3 periodic, tau 0.6, space-time varying phi "
                          f"(T = 1000 steps, refreshed every {K_EPS}), body force 1e-6 x",
              "cells": N, "l2_flush": "inputs larger than L2 (populations 1.27 GB)",
              "parallelism": f"replicas x{world}"}

    if args.impl == "reference":
        if rank != 0:
            return
        cb = cpu_baseline(sample_L=48 if L >= 48 else L, budget_s=max(5.0, args.steps * 0.5), plan=False)
        line = {"impl": "reference", "metric": metric_name(args.size), "value": cb["value"], "unit": "GLUPS",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config, "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")

    res, e2e, tuning = run_gpu(args, rank, world)
    main_st = args.storages[0]
    r = res[main_st]
    glups = aggregate_glups(N, args.steps, r["total_ms"], world)
    peak, peak_kind = peak_hbm()
    bpc = bytes_per_cell(main_st)
    achieved = bpc * N / (r["kernel_ms"] * 1e-3) / 1e9
    src_hash = kernel_source_hash()
    line = {
        "metric": metric_name(args.size), "value": glups, "unit": "GLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["total_ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if main_st == "fp32" else "f16-storage/f32-compute", "data": "synthetic",
        "config": config,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{peak_kind} copy bandwidth",
                     "traffic": profiled_traffic(main_st, src_hash),
                     "algorithmic_bytes_per_cell": bpc,
                     "kernel": r["kernel"], "kernel_ms": r["kernel_ms"],
                     "launch_shape": r["launch_shape"], "tuned_from": r["tuned_from"]},
        "gpu_launches": r["launches"], "clocks": r["clocks"], "e2e": e2e,
    }
    for st, rr in res.items():
        if st == main_st:
            continue
        bb = bytes_per_cell(st)
        ach = bb * N / (rr["kernel_ms"] * 1e-3) / 1e9
        line[st] = {"value": N / (rr["total_ms"] / args.steps) / 1e6, "unit": "GLUPS",
                    "kernel_ms": rr["kernel_ms"], "algorithmic_bytes_per_cell": bb,
                    "achieved_gbs": ach, "frac": ach / peak, "gpu_launches": rr["launches"],
                    "traffic": profiled_traffic(st, src_hash), "clocks": rr["clocks"],
                    "launch_shape": rr["launch_shape"], "tuned_from": rr["tuned_from"]}
    if tuning:
        line["tuning"] = tuning
    if rank == 0 and not args.no_batch:
        line["batched"] = run_batched(args.batch_count, args.batch_steps)
    if rank == 0 and not args.no_porous:
        line["porous_channel"] = run_porous(args.porous_steps)
    if rank == 0 and not args.no_serve:
        line["serving"] = run_serving(tuple(args.serve_rates), args.serve_window)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(sample_L=48 if L >= 48 else L, budget_s=15.0)
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
