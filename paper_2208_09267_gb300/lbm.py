"""ctypes binding of liblbm_vanse.so (include/lbm_vanse.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Host arrays are numpy arrays (copied by the library), device
arrays are CUDA torch tensors (passed by pointer, ``on_device=1``).  There is
no fallback: if the shared library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LATTICES = {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2, "D1Q3": 3}
STORAGES = {"fp64": 0, "fp32": 1, "fp16": 2}
Q_OF = {0: 9, 1: 19, 2: 27, 3: 3}
DIM_OF = {0: 2, 1: 3, 2: 3, 3: 1}
STATUS = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA",
          -4: "LBM_EUNSTABLE", -5: "LBM_ETIMEOUT", -6: "LBM_ESTATE"}

_lock = threading.Lock()
_lib = None


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("storage", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
        ("quad_dim", ctypes.c_int), ("quad_axes", ctypes.c_uint),
        ("walls", ctypes.c_uint), ("fp16_scale_log2", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p), ("hbm_budget_bytes", ctypes.c_size_t),
        ("block_x", ctypes.c_int), ("block_y", ctypes.c_int), ("kernel", ctypes.c_int),
        ("fp16_rounding", ctypes.c_int), ("quad_auto", ctypes.c_int),
        ("drag_model", ctypes.c_int), ("drag_c1", ctypes.c_double), ("drag_c2", ctypes.c_double),
        ("drag_d", ctypes.c_double), ("les_cs", ctypes.c_double),
        ("row_consumers", ctypes.c_int), ("row_stages", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3),
        ("residual", ctypes.c_double), ("u_norm", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("steps_done", ctypes.c_longlong), ("step_of_stats", ctypes.c_longlong),
        ("nan_seen", ctypes.c_int), ("converged", ctypes.c_int),
    ]

    def as_dict(self):
        return {"mass": self.mass, "momentum": tuple(self.momentum), "residual": self.residual,
                "u_norm": self.u_norm, "force": tuple(self.force), "steps_done": self.steps_done,
                "step_of_stats": self.step_of_stats, "nan_seen": bool(self.nan_seen),
                "converged": bool(self.converged)}


# Every function the header declares, with its ctypes signature.
_H = ctypes.c_void_p
_P = ctypes.c_void_p
_SIGS = {
    "lbm_vanse_version": (ctypes.c_char_p, []),
    "lbm_vanse_last_error": (ctypes.c_char_p, [_H]),
    "lbm_vanse_params_default": (ctypes.c_int, [ctypes.POINTER(Params)]),
    "lbm_vanse_device_bytes": (ctypes.c_size_t, [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int]),
    "lbm_vanse_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_vanse_destroy": (None, [_H]),
    "lbm_vanse_set_epsilon": (ctypes.c_int, [_H, _P, _P, ctypes.c_longlong, ctypes.c_int]),
    "lbm_vanse_set_epsilon_f64": (ctypes.c_int, [_H, _P, _P, ctypes.c_longlong, ctypes.c_int]),
    "lbm_vanse_stage_epsilon": (ctypes.c_int, [_H, _P, _P, ctypes.c_longlong, ctypes.c_int]),
    "lbm_vanse_commit_epsilon": (ctypes.c_int, [_H]),
    "lbm_vanse_set_force": (ctypes.c_int, [_H, _P, _P, _P, ctypes.c_longlong, ctypes.c_int]),
    "lbm_vanse_set_force_f64": (ctypes.c_int, [_H, _P, _P, _P, ctypes.c_longlong, ctypes.c_int]),
    "lbm_vanse_init_equilibrium": (ctypes.c_int, [_H, _P, _P, ctypes.c_int, ctypes.c_int]),
    "lbm_vanse_init_equilibrium_f64": (ctypes.c_int, [_H, _P, _P, ctypes.c_int, ctypes.c_int]),
    "lbm_vanse_step": (ctypes.c_int, [_H, ctypes.c_longlong, ctypes.c_double, ctypes.c_int,
                                      ctypes.POINTER(Stats)]),
    "lbm_vanse_moments": (ctypes.c_int, [_H, _P, _P, _P, ctypes.c_int]),
    "lbm_vanse_moments_f64": (ctypes.c_int, [_H, _P, _P, _P, ctypes.c_int]),
    "lbm_vanse_moments_noalloc": (ctypes.c_int, [_H, _P, _P, _P]),
    "lbm_vanse_get_populations": (ctypes.c_int, [_H, _P]),
    "lbm_vanse_steps_done": (ctypes.c_longlong, [_H]),
    "lbm_vanse_launch_count": (ctypes.c_longlong, []),
    "lbm_vanse_set_wait_limit": (ctypes.c_int, [_H, ctypes.c_uint, ctypes.c_int]),
    "lbm_vanse_uses_row_kernel": (ctypes.c_int, [_H]),
    "lbm_vanse_launch_shape": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int * 4)]),
    "lbm_vanse_get_params": (ctypes.c_int, [_H, ctypes.POINTER(Params)]),
    "lbm_vanse_save_state": (ctypes.c_int, [_H, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_vanse_load_state": (ctypes.c_int, [_H, _P, ctypes.c_size_t]),
    "lbm_vanse_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                                              ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_vanse_batch_destroy": (None, [_H]),
    "lbm_vanse_batch_add": (ctypes.c_int, [_H, _H, ctypes.c_longlong]),
    "lbm_vanse_batch_remove": (ctypes.c_int, [_H, _H]),
    "lbm_vanse_batch_step": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int]),
    "lbm_vanse_batch_stats": (ctypes.c_int, [_H, _H, ctypes.POINTER(Stats)]),
    "lbm_vanse_batch_size": (ctypes.c_int, [_H]),
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load the shared library (building it in-tree if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise OSError(f"{path} not found: run paper_2208_09267_gb300.build.build()")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def last_error(h=None) -> str:
    s = lib().lbm_vanse_last_error(h)
    return s.decode() if s else ""


def _check(code, h=None):
    if code != 0:
        raise LbmError(code, last_error(h))
    return code


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _arg(a, n, f64, name):
    """(pointer, on_device, keepalive) for an optional field argument."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        import torch
        want = torch.float64 if f64 else torch.float32
        if not a.is_cuda or a.dtype != want or not a.is_contiguous() or a.numel() != n:
            raise ValueError(f"{name}: expected a contiguous CUDA {want} tensor of {n} values")
        return a.data_ptr(), 1, a
    arr = np.ascontiguousarray(a, dtype=np.float64 if f64 else np.float32)
    if arr.size != n:
        raise ValueError(f"{name}: expected {n} values, got {arr.size}")
    return arr.ctypes.data, 0, arr


def _same_device_kind(*items):
    kinds = {k for _, k, _ in items if k is not None}
    if len(kinds) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return kinds.pop() if kinds else 0


def current_stream_ptr():
    import torch
    return torch.cuda.current_stream().cuda_stream


# limits of lbm_vanse_moments_noalloc (its fixed staging array, 20 bytes per cell)
NOALLOC_SCRATCH_BYTES = 16 << 20
NOALLOC_MAX_CELLS = NOALLOC_SCRATCH_BYTES // 20


def stored_cells(nx: int, ny: int, nz: int) -> int:
    """Cells a lattice holds on the device: every x-row is stored at a pitch
    of nx rounded up to 8 elements (the unit a batch tile counts)."""
    return (nx + 7) // 8 * 8 * ny * nz


class Lattice:
    """One lattice handle (lbm_vanse_t).  Shapes follow the C ABI: fields are
    flat arrays of N = nx*ny*nz values with x fastest; vector fields have
    3*N values, component-major."""

    def __init__(self, lattice="D3Q19", shape=(32, 32, 32), tau=0.6, storage="fp32", rho0=1.0,
                 quad_axes=0, quad_dim=0, walls=0, fp16_scale_log2=10, stream=None,
                 hbm_budget_bytes=0, block=(0, 0), kernel=0, fp16_rounding="stochastic",
                 drag=None, les_cs=0.0, row_shape=None, tuned=True):
        """shape is (nx, ny, nz); nz = 1 for D2Q9, ny = nz = 1 for D1Q3.
        quad_axes: an axis bitmask, 0 (every axis) or "auto" (chosen from
        phi at every refresh).  drag: None or (c1, c2, d) of the Ergun-type
        drag law; les_cs: Smagorinsky constant (0 = BGK).  row_shape:
        (consumer warps, staged rows) of the row-staged kernel, or None.
        tuned: when kernel, block and row_shape are left at their defaults,
        take them from the autotuner's cache for this size bucket (tune.py),
        if it holds an entry."""
        L = lib()
        p = Params()
        _check(L.lbm_vanse_params_default(ctypes.byref(p)))
        self.tuned_from = None
        if tuned and kernel in (0, "auto") and tuple(block) == (0, 0) and row_shape is None:
            from . import tune
            hit = tune.best_config(lattice if isinstance(lattice, str) else
                                   {v: k for k, v in LATTICES.items()}[int(lattice)],
                                   storage if isinstance(storage, str) else
                                   {v: k for k, v in STORAGES.items()}[int(storage)], shape)
            if hit is not None:
                kernel, block, row_shape = hit["kernel"], tuple(hit["block"]), hit.get("row_shape")
                self.tuned_from = hit.get("key")
        p.lattice = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
        p.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
        nx, ny, nz = (list(shape) + [1, 1])[:3]
        p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
        p.tau, p.rho0 = float(tau), float(rho0)
        if isinstance(quad_axes, str):
            if quad_axes != "auto":
                raise ValueError('quad_axes: an axis bitmask or "auto"')
            p.quad_auto, quad_axes = 1, 0
        p.quad_axes, p.quad_dim, p.walls = int(quad_axes), int(quad_dim), int(walls)
        p.fp16_scale_log2 = int(fp16_scale_log2)
        p.cuda_stream = stream
        p.hbm_budget_bytes = int(hbm_budget_bytes)
        p.block_x, p.block_y = int(block[0]), int(block[1])
        p.kernel = {"auto": 0, "cell": 1, "row": 2}.get(kernel, kernel)
        p.fp16_rounding = {"stochastic": 0, "nearest": 1}.get(fp16_rounding, fp16_rounding)
        if row_shape is not None:
            p.row_consumers, p.row_stages = (int(v) for v in row_shape)
        if drag is not None:
            p.drag_model = 1
            p.drag_c1, p.drag_c2, p.drag_d = (float(v) for v in drag)
        p.les_cs = float(les_cs)
        h = ctypes.c_void_p()
        _check(L.lbm_vanse_create(ctypes.byref(p), ctypes.byref(h)))
        self._h = h
        self.params = p
        self.lattice = p.lattice
        self.q = Q_OF[p.lattice]
        self.d = DIM_OF[p.lattice]
        self.nx, self.ny, self.nz = p.nx, p.ny, p.nz
        self.n = p.nx * p.ny * p.nz
        # cells as stored on the device: x-rows padded to a multiple of 8
        self.stored = stored_cells(p.nx, p.ny, p.nz)
        self.f64 = p.storage == 0

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_vanse_destroy(self._h)
            self._h = None
        self._staged = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        if not self._h:
            raise LbmError(-6, "handle is closed")
        return self._h

    # -- inputs -----------------------------------------------------------
    def set_epsilon(self, eps_ref, deps_dt=None, n_ref=0, f64=None):
        f64 = self.f64 if f64 is None else f64
        a = _arg(eps_ref, self.n, f64, "eps_ref")
        b = _arg(deps_dt, self.n, f64, "deps_dt")
        dev = _same_device_kind(a, b)
        fn = lib().lbm_vanse_set_epsilon_f64 if f64 else lib().lbm_vanse_set_epsilon
        _check(fn(self.handle, a[0], b[0], int(n_ref), dev), self.handle)

    def stage_epsilon(self, eps_ref, deps_dt=None, n_ref=0):
        """Start the upload of a phi refresh (FP32 values) on the library's
        copy stream; steps issued before commit_epsilon() overlap it.  The
        arrays are kept alive here until the commit."""
        a = _arg(eps_ref, self.n, False, "eps_ref")
        b = _arg(deps_dt, self.n, False, "deps_dt")
        dev = _same_device_kind(a, b)
        _check(lib().lbm_vanse_stage_epsilon(self.handle, a[0], b[0], int(n_ref), dev), self.handle)
        self._staged = (a[2], b[2])

    def commit_epsilon(self):
        """Make the staged refresh current (as set_epsilon would)."""
        try:
            _check(lib().lbm_vanse_commit_epsilon(self.handle), self.handle)
        finally:
            self._staged = None

    def set_force(self, g=(0.0, 0.0, 0.0), field=None, dfield_dt=None, n_ref=0, f64=None):
        f64 = self.f64 if f64 is None else f64
        gv = (ctypes.c_double * 3)(*[float(v) for v in (list(g) + [0.0] * 3)[:3]])
        a = _arg(field, 3 * self.n, f64, "field")
        b = _arg(dfield_dt, 3 * self.n, f64, "dfield_dt")
        dev = _same_device_kind(a, b)
        fn = lib().lbm_vanse_set_force_f64 if f64 else lib().lbm_vanse_set_force
        _check(fn(self.handle, gv, a[0], b[0], int(n_ref), dev), self.handle)

    def init_equilibrium(self, p0=None, u0=None, integral=False, half_force=False, f64=None):
        f64 = self.f64 if f64 is None else f64
        if u0 is not None and not _is_torch(u0):
            u0 = np.asarray(u0, dtype=np.float64).reshape(-1, self.n)
            u0 = np.vstack([u0, np.zeros((3 - u0.shape[0], self.n))])
        a = _arg(p0, self.n, f64, "p0")
        b = _arg(u0, 3 * self.n, f64, "u0")
        dev = _same_device_kind(a, b)
        mode = (1 if integral else 0) | (2 if half_force else 0)
        fn = lib().lbm_vanse_init_equilibrium_f64 if f64 else lib().lbm_vanse_init_equilibrium
        _check(fn(self.handle, a[0], b[0], mode, dev), self.handle)

    # -- stepping -----------------------------------------------------------
    def step(self, max_steps, residual_tol=0.0, check_every=0):
        st = Stats()
        code = lib().lbm_vanse_step(self.handle, int(max_steps), float(residual_tol),
                                    int(check_every), ctypes.byref(st))
        if code != 0:
            raise LbmError(code, last_error(self.handle))
        return st.as_dict()

    @property
    def quadrature(self):
        """(quad_axes, quad_dim) in use: the axes of eq. (quad) and the row
        of Table "weights" (chosen from phi when created with
        quad_axes="auto")."""
        p = Params()
        _check(lib().lbm_vanse_get_params(self.handle, ctypes.byref(p)), self.handle)
        return int(p.quad_axes), int(p.quad_dim)

    @property
    def launch_shape(self) -> dict:
        """The step's launch shape (kernel and, for the row-staged kernel,
        consumer warps, staged rows and grid)."""
        a = (ctypes.c_int * 4)()
        _check(lib().lbm_vanse_launch_shape(self.handle, ctypes.byref(a)), self.handle)
        kern = {0: "fp64-cell", 1: "cell", 2: "row"}[a[0]]
        if a[0] == 2:
            return {"kernel": kern, "consumers": a[1], "stages": a[2], "grid": a[3]}
        return {"kernel": kern, "block": [a[1], a[2]], "grid": a[3]}

    @property
    def row_kernel(self) -> bool:
        return lib().lbm_vanse_uses_row_kernel(self.handle) == 1

    def set_wait_limit(self, spins: int, withhold_copies: bool = False):
        _check(lib().lbm_vanse_set_wait_limit(self.handle, int(spins), int(bool(withhold_copies))),
               self.handle)

    @property
    def steps_done(self):
        return int(lib().lbm_vanse_steps_done(self.handle))

    # -- outputs ------------------------------------------------------------
    def moments(self, f64=True):
        """dict(rho, p, u) as numpy arrays: (N,), (N,), (3, N)."""
        dt = np.float64 if f64 else np.float32
        rho = np.empty(self.n, dt)
        p = np.empty(self.n, dt)
        u = np.empty(3 * self.n, dt)
        fn = lib().lbm_vanse_moments_f64 if f64 else lib().lbm_vanse_moments
        _check(fn(self.handle, rho.ctypes.data, p.ctypes.data, u.ctypes.data, 0), self.handle)
        return {"rho": rho, "p": p, "u": u.reshape(3, self.n)}

    def moments_noalloc(self):
        """dict(rho, p, u) as float32 numpy arrays, read back through the
        library's fixed staging array instead of a temporary device buffer
        (lattices of at most NOALLOC_MAX_CELLS cells; concurrent calls from
        several threads must be serialised by the caller)."""
        rho = np.empty(self.n, np.float32)
        p = np.empty(self.n, np.float32)
        u = np.empty(3 * self.n, np.float32)
        _check(lib().lbm_vanse_moments_noalloc(self.handle, rho.ctypes.data, p.ctypes.data,
                                               u.ctypes.data), self.handle)
        return {"rho": rho, "p": p, "u": u.reshape(3, self.n)}

    def moments_into(self, rho=None, p=None, u=None):
        """Write moments into CUDA float32/float64 torch tensors (stream-ordered)."""
        items = [t for t in (rho, p, u) if t is not None]
        f64 = items[0].dtype.__repr__().endswith("float64") if items else False
        ptrs = []
        for t, n, name in ((rho, self.n, "rho"), (p, self.n, "p"), (u, 3 * self.n, "u")):
            ptrs.append(_arg(t, n, f64, name)[0])
        fn = lib().lbm_vanse_moments_f64 if f64 else lib().lbm_vanse_moments
        _check(fn(self.handle, ptrs[0], ptrs[1], ptrs[2], 1), self.handle)

    def populations(self):
        """Decoded f_i(x, n), shape (N, Q), float64, natural order."""
        f = np.empty((self.n, self.q), np.float64)
        _check(lib().lbm_vanse_get_populations(self.handle, f.ctypes.data), self.handle)
        return f

    def save_state(self) -> bytes:
        size = ctypes.c_size_t(0)
        _check(lib().lbm_vanse_save_state(self.handle, None, ctypes.byref(size)), self.handle)
        buf = ctypes.create_string_buffer(size.value)
        _check(lib().lbm_vanse_save_state(self.handle, buf, ctypes.byref(size)), self.handle)
        return buf.raw[: size.value]

    def load_state(self, state: bytes):
        buf = ctypes.create_string_buffer(state, len(state))
        _check(lib().lbm_vanse_load_state(self.handle, buf, len(state)), self.handle)


def device_bytes(lattice="D3Q19", shape=(32, 32, 32), storage="fp32", with_deps=False,
                 with_force_field=False, block=(0, 0)) -> int:
    L = lib()
    p = Params()
    _check(L.lbm_vanse_params_default(ctypes.byref(p)))
    p.lattice = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    p.storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
    nx, ny, nz = (list(shape) + [1, 1])[:3]
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    p.block_x, p.block_y = int(block[0]), int(block[1])
    return int(L.lbm_vanse_device_bytes(ctypes.byref(p), int(with_deps), int(with_force_field)))


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().lbm_vanse_launch_count())


def version() -> str:
    return lib().lbm_vanse_version().decode()


class Batch:
    """Many lattices advanced together (lbm_vanse_batch_t): one persistent,
    graph-captured kernel per (lattice, storage) type per step."""

    def __init__(self, max_members=256, max_tiles=65536, tile_cells=None, stream=None, storage="fp16"):
        """tile_cells: cells per tile of the one-cell-per-thread batch kernel;
        None = the autotuner's cached choice for this storage, else the
        library default."""
        self.tuned_from = None
        if tile_cells is None:
            from . import tune
            hit = tune.best_tile(storage)
            tile_cells = hit["best"] if hit else 0
            self.tuned_from = hit["key"] if hit else None
        self.tile_cells = int(tile_cells)
        h = ctypes.c_void_p()
        _check(lib().lbm_vanse_batch_create(int(max_members), int(max_tiles), int(tile_cells),
                                            stream, ctypes.byref(h)))
        self._h = h
        self.members = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_vanse_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, lat: Lattice, max_steps: int) -> int:
        slot = lib().lbm_vanse_batch_add(self._h, lat.handle, int(max_steps))
        if slot < 0:
            raise LbmError(slot, last_error())
        self.members[id(lat)] = lat
        return slot

    def remove(self, lat: Lattice):
        _check(lib().lbm_vanse_batch_remove(self._h, lat.handle))
        self.members.pop(id(lat), None)

    def step(self, k: int, check: bool = False):
        _check(lib().lbm_vanse_batch_step(self._h, int(k), int(bool(check))))

    def stats(self, lat: Lattice) -> dict:
        st = Stats()
        _check(lib().lbm_vanse_batch_stats(self._h, lat.handle, ctypes.byref(st)))
        return st.as_dict()

    def __len__(self):
        return int(lib().lbm_vanse_batch_size(self._h))
