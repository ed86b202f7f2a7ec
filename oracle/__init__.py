"""FP64 CPU oracle of the consistent VANSE lattice Boltzmann scheme.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain reference that the
CUDA library is checked against (Bukreev et al., arXiv 2208.09267, Sec. 2.2).
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product path never does.  It shares no code
with the CUDA path: the arithmetic lives in ``lbm_oracle.c`` (plain C, FP64,
compiled with ``-ffp-contract=off``), this module only marshals numpy arrays.

Every function here is pinned by ``tests/test_oracle_*.py`` against what the
paper and the mathematics fix (weights of Tables "latt_par", "latt_3d" and
"weights", the moment identities of eqs. (M0)-(M3) and (M0F)-(M2F), the
epsilon == 1 reduction to plain BGK with Guo forcing, conservation, Poiseuille
closed forms and the second-order convergence of Sec. 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

LATTICES = {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2, "D1Q3": 3}
Q_OF = {0: 9, 1: 19, 2: 27, 3: 3}
DIM_OF = {0: 2, 1: 3, 2: 3, 3: 1}


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into oracle/_build/liblbm_oracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
        ("quad_dim", ctypes.c_int), ("quad_axes", ctypes.c_uint),
        ("walls", ctypes.c_uint),
        ("eps_ref", ctypes.c_void_p), ("deps_dt", ctypes.c_void_p),
        ("n_eps", ctypes.c_longlong),
        ("g", ctypes.c_double * 3),
        ("force", ctypes.c_void_p), ("dforce_dt", ctypes.c_void_p),
        ("n_force", ctypes.c_longlong),
        ("drag_model", ctypes.c_int),
        ("drag_c1", ctypes.c_double), ("drag_c2", ctypes.c_double), ("drag_d", ctypes.c_double),
        ("les_cs", ctypes.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Problem)
            dp = ctypes.c_void_p
            _lib.oracle_step.argtypes = [P, ctypes.c_longlong, dp, dp]
            _lib.oracle_run.argtypes = [P, ctypes.c_longlong, ctypes.c_longlong, dp, dp]
            _lib.oracle_run_series.argtypes = [P, ctypes.c_longlong, ctypes.c_longlong,
                                               dp, dp, dp, dp]
            _lib.oracle_init.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_longlong, dp]
            _lib.oracle_moments.argtypes = [P, ctypes.c_longlong, dp, dp, dp, dp, dp]
            _lib.oracle_forces.argtypes = [P, ctypes.c_longlong, dp, dp]
            _lib.oracle_cell_terms.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp,
                                               ctypes.c_double, dp, dp]
            _lib.oracle_velocity_set.argtypes = [ctypes.c_int, dp, dp, dp]
            _lib.oracle_quad_weights.argtypes = [ctypes.c_int, dp]
            _lib.oracle_set_threads.argtypes = [ctypes.c_int]
            _lib.oracle_q.argtypes = [ctypes.c_int]
        return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def set_threads(n: int) -> None:
    """Number of OpenMP threads for oracle_step (0 = all cores)."""
    lib().oracle_set_threads(int(n))


def velocity_set(lattice: int):
    """(c[Q,3], w[Q], opp[Q]) of the oracle's own velocity tables."""
    q = Q_OF[lattice]
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    opp = np.zeros(q, dtype=np.int32)
    lib().oracle_velocity_set(lattice, c.ctypes.data, w.ctypes.data, opp.ctypes.data)
    return c, w, opp


def quad_weights(quad_dim: int):
    w = np.zeros(2)
    if lib().oracle_quad_weights(quad_dim, w.ctypes.data):
        raise ValueError("quad_dim must be 1, 2, 3 or -1 (pointwise)")
    return w


def quadrature_axes(eps_ref, deps_dt=None, dims=3):
    """The quadrature rule of Sec. 2.2, chosen by how many axes phi varies
    along: (quad_axes, quad_dim) with bit a set when phi_ref (or
    d_t phi) differs anywhere from its periodic neighbour along axis a < dims
    (exact comparison), and every axis when phi is uniform.  Fields have
    shape (nz, ny, nx)."""
    mask = 0
    for f in (eps_ref, deps_dt):
        if f is None:
            continue
        f = np.asarray(f)
        for a in range(dims):
            if np.any(np.roll(f, -1, axis=2 - a) != f):
                mask |= 1 << a
    if mask == 0:
        mask = (1 << dims) - 1
    return mask, bin(mask).count("1")


def cell_terms(lattice: int, M0: float, u, F, tau: float):
    """(f^eq[Q], Omega^F[Q]) of one cell (eq. (feq) and the Guo term)."""
    q = Q_OF[lattice]
    u = _f64(np.pad(np.asarray(u, float), (0, 3 - len(u))))
    F = _f64(np.pad(np.asarray(F, float), (0, 3 - len(F))))
    feq = np.zeros(q)
    om = np.zeros(q)
    lib().oracle_cell_terms(lattice, M0, u.ctypes.data, F.ctypes.data, tau,
                            feq.ctypes.data, om.ctypes.data)
    return feq, om


class Problem:
    """One lattice problem for the oracle.

    Fields are numpy arrays with x fastest: ``eps_ref`` has shape
    (nz, ny, nx) (nz = 1 in 2D); ``force`` has shape (3, nz, ny, nx).
    Populations are AoS float64 arrays of shape (N, Q).
    """

    def __init__(self, lattice, nx, ny, nz=1, tau=0.8, rho0=1.0, quad_dim=None,
                 quad_axes=None, walls=0, eps_ref=None, deps_dt=None, n_eps=0,
                 g=(0.0, 0.0, 0.0), force=None, dforce_dt=None, n_force=0, drag=None,
                 les_cs=0.0):
        """drag: None, or (c1, c2, d) of the Ergun-type drag law (R9 of
        lbm_oracle.c); les_cs: Smagorinsky constant (R10), 0 = BGK."""
        if isinstance(lattice, str):
            lattice = LATTICES[lattice]
        self.lattice = lattice
        self.q = Q_OF[lattice]
        self.d = DIM_OF[lattice]
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        self.nx, self.ny, self.nz = nx, ny, nz
        self.tau, self.rho0 = float(tau), float(rho0)
        if quad_axes is None:
            quad_axes = (1 << self.d) - 1
        if quad_dim is None:
            quad_dim = bin(quad_axes).count("1")
        self.quad_dim, self.quad_axes, self.walls = quad_dim, quad_axes, walls
        self.g = tuple(float(v) for v in (list(g) + [0.0] * 3)[:3])
        self.drag = None if drag is None else tuple(float(v) for v in drag)
        self.les_cs = float(les_cs)
        self.set_epsilon(np.ones(self.shape) if eps_ref is None else eps_ref, deps_dt, n_eps)
        self.set_force(self.g, force, dforce_dt, n_force)

    def set_epsilon(self, eps_ref, deps_dt=None, n_eps=0):
        self.eps_ref = _f64(eps_ref, self.n)
        self.deps_dt = _f64(deps_dt, self.n)
        self.n_eps = int(n_eps)

    def set_force(self, g=None, force=None, dforce_dt=None, n_force=0):
        if g is not None:
            self.g = tuple(float(v) for v in (list(g) + [0.0] * 3)[:3])
        self.force = _f64(force, 3 * self.n)
        self.dforce_dt = _f64(dforce_dt, 3 * self.n)
        self.n_force = int(n_force)

    def _c(self):
        p = _Problem()
        p.lattice = self.lattice
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        p.tau, p.rho0 = self.tau, self.rho0
        p.quad_dim, p.quad_axes, p.walls = self.quad_dim, self.quad_axes, self.walls
        p.eps_ref = _ptr(self.eps_ref)
        p.deps_dt = _ptr(self.deps_dt)
        p.n_eps = self.n_eps
        p.g = (ctypes.c_double * 3)(*self.g)
        p.force = _ptr(self.force)
        p.dforce_dt = _ptr(self.dforce_dt)
        p.n_force = self.n_force
        if self.drag is not None:
            p.drag_model = 1
            p.drag_c1, p.drag_c2, p.drag_d = self.drag
        p.les_cs = self.les_cs
        return p

    def init(self, p0=None, u0=None, with_integral=False, half_force=False, n=0):
        f = np.zeros((self.n, self.q))
        p0 = _f64(p0, self.n)
        if u0 is not None:
            u0 = np.asarray(u0, dtype=np.float64).reshape(-1, self.n)
            u0 = _f64(np.vstack([u0, np.zeros((3 - u0.shape[0], self.n))]), 3 * self.n)
        if lib().oracle_init(ctypes.byref(self._c()), _ptr(p0), _ptr(u0),
                             int(bool(with_integral)) | (2 if half_force else 0),
                             int(n), f.ctypes.data):
            raise ValueError("oracle_init rejected the problem")
        return f

    def step(self, f, n):
        out = np.zeros_like(f)
        if lib().oracle_step(ctypes.byref(self._c()), int(n), f.ctypes.data, out.ctypes.data):
            raise ValueError("oracle_step rejected the problem")
        return out

    def run(self, f, n0, nsteps):
        """Advance f (in place copy returned) by nsteps from time n0."""
        f = np.ascontiguousarray(f, dtype=np.float64).copy()
        work = np.empty_like(f)
        if lib().oracle_run(ctypes.byref(self._c()), int(n0), int(nsteps),
                            f.ctypes.data, work.ctypes.data):
            raise ValueError("oracle_run rejected the problem")
        return f

    def run_series(self, f, n0, eps_series=None, force_series=None):
        """Advance f by len(series) steps from time n0 with exact per-step
        phi (shape (steps, N)) and force fields (shape (steps, 3, N))."""
        f = np.ascontiguousarray(f, dtype=np.float64).copy()
        work = np.empty_like(f)
        series = eps_series if eps_series is not None else force_series
        nsteps = len(series)
        es = None if eps_series is None else _f64(eps_series, nsteps * self.n)
        fs = None if force_series is None else _f64(force_series, nsteps * 3 * self.n)
        if lib().oracle_run_series(ctypes.byref(self._c()), int(n0), int(nsteps),
                                   _ptr(es), _ptr(fs), f.ctypes.data, work.ctypes.data):
            raise ValueError("oracle_run_series rejected the problem")
        return f

    def moments(self, f, n):
        """dict(rho, p, u[3], M0) at time n, each shaped like the lattice."""
        rho = np.zeros(self.n)
        p = np.zeros(self.n)
        u = np.zeros(3 * self.n)
        M0 = np.zeros(self.n)
        if lib().oracle_moments(ctypes.byref(self._c()), int(n), f.ctypes.data,
                                rho.ctypes.data, p.ctypes.data, u.ctypes.data,
                                M0.ctypes.data):
            raise ValueError("oracle_moments rejected the problem")
        return {"rho": rho.reshape(self.shape), "p": p.reshape(self.shape),
                "u": u.reshape((3,) + self.shape), "M0": M0.reshape(self.shape)}

    def forces(self, f, n):
        F = np.zeros(3 * self.n)
        if lib().oracle_forces(ctypes.byref(self._c()), int(n), f.ctypes.data, F.ctypes.data):
            raise ValueError("oracle_forces rejected the problem")
        return F.reshape((3,) + self.shape)
