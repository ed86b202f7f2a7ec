"""Autotuner for the step kernels' launch shapes.

For the single-lattice step it sweeps thread-block shapes (bx, by) with
bx*by <= 256; for the batched step it sweeps the tile size (cells per work
item).  Each candidate is timed with CUDA events over a few steps after a
warm-up, on the stream the library launches on.  Results are cached in a
JSON file keyed by (lattice, storage, size bucket), so a shape is measured
once per bucket and reused: the bucket of a lattice is
floor(log2(cells)), and the key also carries nx's residue modulo 32 class
(multiple of 32 or not), which decides how full the x-blocks are.
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import lbm

BLOCK_CANDIDATES = [(32, 1), (32, 2), (32, 4), (32, 8), (64, 1), (64, 2), (64, 4), (128, 1),
                    (128, 2), (256, 1)]
TILE_CANDIDATES = [1024, 2048, 4096, 8192, 16384]
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build",
                             "autotune.json")
# results of tuning runs on GB300 shipped with the package: read first, then
# overlaid by the local cache (which every tuning run writes)
SEED_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_gb300.json")
_lock = threading.Lock()


def bucket_key(lattice: str, storage: str, shape) -> str:
    nx, ny, nz = (list(shape) + [1, 1])[:3]
    cells = nx * ny * nz
    return f"{lattice}/{storage}/b{int(math.log2(max(cells, 1)))}/x{'32' if nx % 32 == 0 else 'r'}"


def default_cache_path() -> str:
    """LBM_TUNE_CACHE, else the package's build directory."""
    return os.environ.get("LBM_TUNE_CACHE") or DEFAULT_CACHE


class Cache:
    def __init__(self, path: str | None = None, seed: str | None = SEED_CACHE):
        path = path or default_cache_path()
        self.path = path
        self.data = {}
        for f in ([seed] if seed else []) + [path]:
            if os.path.exists(f):
                try:
                    with open(f) as fh:
                        self.data.update(json.load(fh))
                except (OSError, ValueError):
                    pass

    def get(self, key):
        return self.data.get(key)

    def put(self, key, value):
        with _lock:
            self.data[key] = value
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            tmp = self.path + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(self.data, fh, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def _time_steps(lat, steps, warmup):
    import torch
    stream = torch.cuda.current_stream()
    lat.step(warmup)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    lat.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


# (consumer warps, staged rows) of the row-staged kernel; shapes the
# library cannot launch for a lattice type fall back to its default and are
# recorded under the shape that ran
ROW_SHAPES = [(0, 0), (3, 2), (4, 2), (4, 3), (5, 2), (5, 3), (6, 2), (6, 3), (7, 2), (7, 3), (11, 3), (13, 4),
              (15, 4)]


def tune_step(lattice="D3Q19", storage="fp32", shape=(128, 128, 128), tau=0.6, steps=20, warmup=4,
              cache: Cache | None = None, blocks=None, row_shapes=None, force=True):
    """Time the row-staged kernel in each shape (consumer warps, staged
    rows) when the lattice qualifies, and the one-cell-per-thread kernel
    with each block shape, on a lattice of this size.  Caches and returns
    (best, timings): best = {"kernel": 1|2, "block": [bx, by], "row_shape":
    [consumers, stages] or None}, timings in ms per step per candidate."""
    import torch
    cache = cache or Cache()
    key = "step/" + bucket_key(lattice, storage, shape)
    hit = cache.get(key)
    if hit and not force:
        return hit["best"], hit["ms"]
    stream = torch.cuda.current_stream().cuda_stream
    nx, ny, nz = (list(shape) + [1, 1])[:3]
    timings, configs = {}, {}

    def trial(kernel, block, row_shape):
        try:
            lat = lbm.Lattice(lattice, (nx, ny, nz), tau=tau, storage=storage, stream=stream,
                              block=block, kernel=kernel, row_shape=row_shape, tuned=False)
        except lbm.LbmError:
            return
        ls = lat.launch_shape
        if ls["kernel"] == "row":
            name = f"row{ls['consumers']}x{ls['stages']}"
            cfg = {"kernel": 2, "block": [0, 0], "row_shape": [ls["consumers"], ls["stages"]]}
        else:
            name = f"cell{ls['block'][0]}x{ls['block'][1]}"
            cfg = {"kernel": 1, "block": list(ls["block"]), "row_shape": None}
        if name not in timings:
            lat.set_force((1e-6, 0, 0))
            lat.init_equilibrium()
            timings[name] = _time_steps(lat, steps, warmup)
            configs[name] = cfg
        lat.close()
    if storage != "fp64":
        for rs in row_shapes or ROW_SHAPES:
            trial(2, (0, 0), rs)
    for bx, by in blocks or BLOCK_CANDIDATES:
        if by > ny or bx > 2 * max(nx, 32):
            continue
        trial(1, (bx, by), None)
    best = min(timings, key=timings.get)
    cache.put(key, {"best": configs[best], "ms": timings, "shape": [nx, ny, nz]})
    return configs[best], timings


def best_config(lattice, storage, shape, cache: Cache | None = None):
    """The cached launch configuration for this size bucket: a dict with
    "kernel" (1 one cell per thread, 2 row-staged), "block" and "row_shape"
    (consumer warps, staged rows), and "key", or None when the bucket has
    not been tuned (the library then chooses)."""
    cache = cache or Cache()
    key = "step/" + bucket_key(lattice, storage, shape)
    hit = cache.get(key)
    if not hit:
        return None
    out = dict(hit["best"])
    out["key"] = key
    return out


def best_tile(storage, cache: Cache | None = None):
    """The cached tile size of the one-cell-per-thread batch kernel for this
    storage ({"best": cells, "key": ...}), or None."""
    cache = cache or Cache()
    keys = sorted(k for k in cache.data if k.startswith(f"tile/{storage}/"))
    if not keys:
        return None
    return {"best": cache.data[keys[-1]]["best"], "key": keys[-1]}


def tune_block(lattice="D3Q19", storage="fp32", shape=(128, 128, 128), tau=0.6, steps=20,
               warmup=4, cache: Cache | None = None, candidates=None, eps=None, force=True):
    """Time each block shape of the one-cell-per-thread kernel on a lattice
    of this size; return the best (bx, by) and the per-candidate ms/step."""
    import torch
    cache = cache or Cache()
    key = "block/" + bucket_key(lattice, storage, shape)
    hit = cache.get(key)
    if hit and not force:
        return tuple(hit["best"]), hit["ms"]
    stream = torch.cuda.current_stream().cuda_stream
    nx, ny, nz = (list(shape) + [1, 1])[:3]
    timings = {}
    for bx, by in candidates or BLOCK_CANDIDATES:
        if by > ny or bx > 2 * max(nx, 32):
            continue
        lat = lbm.Lattice(lattice, (nx, ny, nz), tau=tau, storage=storage, stream=stream,
                          block=(bx, by), kernel="cell", tuned=False)
        if eps is not None:
            lat.set_epsilon(eps)
        lat.set_force((1e-6, 0, 0))
        lat.init_equilibrium()
        timings[f"{bx}x{by}"] = _time_steps(lat, steps, warmup)
        lat.close()
    best = min(timings, key=timings.get)
    bx, by = (int(v) for v in best.split("x"))
    cache.put(key, {"best": [bx, by], "ms": timings, "shape": [nx, ny, nz]})
    return (bx, by), timings


def best_block(lattice, storage, shape, cache: Cache | None = None):
    """Cached block shape for this bucket, or (0, 0) (library default)."""
    cache = cache or Cache()
    hit = cache.get("block/" + bucket_key(lattice, storage, shape))
    return tuple(hit["best"]) if hit else (0, 0)


def tune_tiles(specs, storage="fp16", steps=10, candidates=None, cache: Cache | None = None,
               force=True):
    """Time batched replays of the given lattice specs for each tile size."""
    import torch
    from . import inputs
    cache = cache or Cache()
    key = f"tile/{storage}/n{len(specs)}"
    hit = cache.get(key)
    if hit and not force:
        return hit["best"], hit["ms"]
    stream = torch.cuda.current_stream().cuda_stream
    lats = []
    for s in specs:
        nz, ny, nx = s.shape
        lat = lbm.Lattice(s.lattice, (nx, ny, nz), tau=s.tau, storage=storage, stream=stream,
                          tuned=False)
        lat.set_epsilon(s.eps().ravel())
        lat.set_force(s.g)
        lat.init_equilibrium()
        lats.append(lat)
    timings = {}
    for tc in candidates or TILE_CANDIDATES:
        b = lbm.Batch(max_members=len(lats), max_tiles=sum(
            (lt.stored + tc - 1) // tc for lt in lats) + 1, tile_cells=tc, stream=stream,
            storage=storage)
        for lt in lats:
            b.add(lt, 10 ** 9)
        b.step(2)
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(torch.cuda.current_stream())
        b.step(steps)
        e.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        timings[str(tc)] = a.elapsed_time(e) / steps
        b.close()
    for lt in lats:
        lt.close()
    best = int(min(timings, key=timings.get))
    cache.put(key, {"best": best, "ms": timings})
    del inputs
    return best, timings
