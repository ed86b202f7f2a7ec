"""Seeded synthetic inputs for the VANSE lattice Boltzmann solver.

This module is the only code that both the CUDA path's tests and the FP64
oracle consume.  It produces input arrays only -- volume-fraction fields,
force fields, manufactured solutions, request traces -- and holds none of the
lattice Boltzmann arithmetic (no equilibrium, no moments, no collision).

Workloads (lattice units unless stated):

* ``eps_static_sine``       -- phi = 0.8 + 0.1 sin(2 pi x/n) sin(2 pi y/n): a 64^2
  D2Q9 periodic case with uniform body force.
* ``eps_travelling_wave``   -- phi = 0.7 + 0.2 sin(2 pi x/L) cos(2 pi y/L)
  sin(2 pi z/L + 2 pi t/T), with its analytic time derivative: the space-time
  varying D3Q19 case.
* ``eps_random_spheres``    -- seeded random spheres smoothed by a Gaussian into
  phi in [0.4, 1]: a porous channel with walls on y.
* ``eps_product_sine``      -- phi = (1-a) + a prod_k sin(2 pi x_k/n): the
  per-lattice fields of the batched and served workloads.
* ``MMS`` -- the manufactured solutions of Sec. 3 (Examples 1-5) with the
  manufactured force of Sec. 3 evaluated by central finite differences, as
  the paper does, and the conversion to lattice units under diffusive
  scaling (Sec. 3, physical set-up).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 20220819
CS2 = 1.0 / 3.0


def _xp(a):
    """numpy, or torch when `a` is a torch tensor (the manufactured fields
    below are evaluated with either, so that the GPU tests can generate them
    on the device)."""
    if type(a).__module__.startswith("torch"):
        import torch
        return torch
    return np


def rng(offset: int = 0) -> np.random.Generator:
    return np.random.default_rng(MASTER_SEED + int(offset))


def _grid(shape):
    """Index grids (x, y, z) for a (nz, ny, nx) array, x fastest."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


# --------------------------------------------------------------------------
# Volume-fraction fields
# --------------------------------------------------------------------------

def eps_static_sine(n: int = 64, mean: float = 0.8, amp: float = 0.1) -> np.ndarray:
    """phi(x,y) = mean + amp sin(2 pi x/n) sin(2 pi y/n) on an n x n lattice, (1,n,n)."""
    x, y, _ = _grid((1, n, n))
    return mean + amp * np.sin(2 * np.pi * x / n) * np.sin(2 * np.pi * y / n)


def eps_travelling_wave(L: int, t: float, T: float = 1000.0, mean: float = 0.7,
                        amp: float = 0.2, shape=None):
    """phi and d_t phi of the space-time varying field at step t.

    phi = mean + amp sin(2 pi x/L) cos(2 pi y/L) sin(2 pi z/L + 2 pi t/T).
    Returns (phi, dphi_dt) as float64 arrays shaped (L, L, L).
    """
    shape = shape or (L, L, L)
    x, y, z = _grid(shape)
    a = amp * np.sin(2 * np.pi * x / L) * np.cos(2 * np.pi * y / L)
    ph = 2 * np.pi * z / L + 2 * np.pi * t / T
    return mean + a * np.sin(ph), a * np.cos(ph) * (2 * np.pi / T)


def eps_travelling_wave_torch(L: int, t: float, T: float = 1000.0, mean: float = 0.7,
                              amp: float = 0.2, device="cuda", dtype=None):
    """eps_travelling_wave evaluated with torch on `device` (FP64, then cast
    to `dtype`): flat (phi, d_t phi) of L^3 cells, x fastest."""
    import torch
    dtype = dtype or torch.float64
    k = 2 * np.pi / L
    r = torch.arange(L, dtype=torch.float64, device=device) * k
    sx, cy = torch.sin(r), torch.cos(r)
    ph = r + 2 * np.pi * t / T
    a = (sx.reshape(1, 1, L) * cy.reshape(1, L, 1)) * amp
    e = mean + a * torch.sin(ph).reshape(L, 1, 1)
    d = a * torch.cos(ph).reshape(L, 1, 1) * (2 * np.pi / T)
    return e.reshape(-1).to(dtype).contiguous(), d.reshape(-1).to(dtype).contiguous()


def eps_product_sine(shape, amp: float) -> np.ndarray:
    """phi = (1 - amp) + amp prod_k sin(2 pi x_k / n_k) over the lattice's axes."""
    nz, ny, nx = shape
    x, y, z = _grid(shape)
    s = np.sin(2 * np.pi * x / nx) * np.sin(2 * np.pi * y / ny)
    if nz > 1:
        s = s * np.sin(2 * np.pi * z / nz)
    return (1.0 - amp) + amp * s


def _gauss_kernel1d(sigma: float) -> np.ndarray:
    r = int(math.ceil(3 * sigma))
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / sigma) ** 2)
    return k / k.sum()


def _smooth_axis(a: np.ndarray, k: np.ndarray, axis: int, periodic: bool) -> np.ndarray:
    r = (len(k) - 1) // 2
    out = np.zeros_like(a)
    n = a.shape[axis]
    for j, kj in enumerate(k):
        s = j - r
        if periodic:
            out += kj * np.roll(a, -s, axis=axis)
        else:
            idx = np.arange(n) + s
            idx = np.where(idx < 0, -idx - 1, idx)          # reflect
            idx = np.where(idx >= n, 2 * n - idx - 1, idx)
            out += kj * np.take(a, idx, axis=axis)
    return out


def eps_random_spheres(shape, seed_offset: int = 3, rmin: float = 4.0, rmax: float = 12.0,
                       packing: float = 0.35, sigma: float = 3.0, eps_min: float = 0.4,
                       wall_axis: int | None = 1, max_spheres: int = 1_000_000) -> np.ndarray:
    """Porous field: random spheres (radius U[rmin, rmax], overlap allowed) are
    added until the solid fraction of the union reaches ``packing``; the
    indicator is smoothed by a normalised Gaussian (sigma cells, cut at
    3 sigma; periodic on the non-wall axes, reflecting on the wall axis) and
    mapped to phi = 1 - (1 - eps_min) G*chi in [eps_min, 1].

    With ``wall_axis`` set, the first and last layer on that axis are wall
    layers: they hold the phi of their fluid neighbour.
    """
    nz, ny, nx = shape
    g = rng(seed_offset)
    chi = np.zeros(shape, dtype=np.float32)
    ntot = chi.size
    solid = 0
    x = np.arange(nx)
    y = np.arange(ny)
    z = np.arange(nz)
    count = 0
    flat = nz == 1          # a 2D lattice: the spheres become disks in z = 0
    while solid < packing * ntot and count < max_spheres:
        c = g.uniform(0, 1, 3) * np.array([nx, ny, nz])
        if flat:
            c[2] = 0.0
        r = g.uniform(rmin, rmax)
        count += 1
        # bounding box (periodic on every axis except the wall axis)
        sl = []
        for ax_len, cc, ax in ((nz, c[2], 0), (ny, c[1], 1), (nx, c[0], 2)):
            lo, hi = int(math.floor(cc - r)), int(math.ceil(cc + r)) + 1
            idx = np.arange(lo, hi)
            axis_id = {0: 2, 1: 1, 2: 0}[ax]          # (z,y,x) -> lattice axis id
            if ax == 0 and flat:
                idx = np.array([0])
            # a box wider than the lattice would repeat indices in the scatter
            if len(idx) > ax_len:
                idx = idx[:ax_len]
            if wall_axis is not None and axis_id == wall_axis:
                idx = idx[(idx >= 0) & (idx < ax_len)]
            sl.append(idx)
        iz, iy, ix = sl
        if len(iz) == 0 or len(iy) == 0 or len(ix) == 0:
            continue
        dz = (iz - c[2])[:, None, None]
        dy = (iy - c[1])[None, :, None]
        dx = (ix - c[0])[None, None, :]
        inside = (dx * dx + dy * dy + dz * dz) <= r * r
        zz, yy, xx = np.mod(iz, nz), np.mod(iy, ny), np.mod(ix, nx)
        blk = chi[np.ix_(zz, yy, xx)]
        newly = inside & (blk == 0)
        solid += int(newly.sum())
        blk[inside] = 1.0
        chi[np.ix_(zz, yy, xx)] = blk
    k = _gauss_kernel1d(sigma)
    a = chi.astype(np.float64)
    for axis, lattice_axis in ((2, 0), (1, 1), (0, 2)):
        if a.shape[axis] > 1:
            a = _smooth_axis(a, k, axis, periodic=(wall_axis != lattice_axis))
    eps = 1.0 - (1.0 - eps_min) * a
    if wall_axis is not None:
        eps = np.moveaxis(eps, 2 - wall_axis, 0).copy()
        eps[0] = eps[1]
        eps[-1] = eps[-2]
        eps = np.moveaxis(eps, 0, 2 - wall_axis)
    return np.ascontiguousarray(eps)


# --------------------------------------------------------------------------
# Manufactured solutions of Sec. 3
# --------------------------------------------------------------------------

def _d(fun, axis: int, h: float = 1e-3):
    """Sixth-order central difference of fun(X, t) along coordinate ``axis``
    (axis 3 = time)."""
    def dfun(X, t):
        def shifted(s):
            if axis == 3:
                return fun(X, t + s * h)
            Y = list(X)
            Y[axis] = X[axis] + s * h
            return fun(Y, t)
        return (45.0 * (shifted(1) - shifted(-1)) - 9.0 * (shifted(2) - shifted(-2))
                + (shifted(3) - shifted(-3))) / (60.0 * h)
    return dfun


@dataclass
class MMS:
    """Manufactured solution ``example`` (1..5) of Sec. 3 on the periodic box
    [0, 2 m]^d with N nodes per axis, rho = 1, nu = 0.1 m^2/s, and tau = 0.53
    (stationary, Examples 1-2) or 0.5075 (transient, Examples 3-5) held fixed
    under diffusive scaling.

    Example 5 reading: the printed fields carry no time dependence and then
    violate the mass equation (vansEquMass); the travelling-wave argument
    pi (x_k - 0.5 t) of Examples 3-4 is used in every factor instead.
    Example 3 (one-dimensional) runs on a D2Q9 lattice of N x 1 nodes.
    """
    example: int
    N: int
    length: float = 2.0
    nu: float = 0.1
    tau: float | None = None
    h_fd: float = 1e-3
    lattice: str = field(init=False)
    dim: int = field(init=False)

    def __post_init__(self):
        if self.example not in (1, 2, 3, 4, 5):
            raise ValueError("example must be 1..5")
        self.stationary = self.example in (1, 2)
        if self.tau is None:
            self.tau = 0.53 if self.stationary else 0.5075
        self.dim = {1: 2, 2: 3, 3: 1, 4: 2, 5: 3}[self.example]
        self.lattice = "D3Q27" if self.dim == 3 else "D2Q9"
        self.dx = self.length / self.N
        self.nu_lattice = (self.tau - 0.5) * CS2
        self.dt = self.nu_lattice * self.dx * self.dx / self.nu
        n = self.N
        self.shape = (n, n, n) if self.dim == 3 else ((1, n, n) if self.dim == 2 else (1, 1, n))
        self.quad_axes = {1: 1, 2: 3, 3: 7}[self.dim]

    # analytic fields, X = (x, y, z) in metres, t in seconds
    def eps(self, X, t):
        x, y, z = X
        s = _xp(x).sin
        pi = np.pi
        e = self.example
        if e == 1:
            return 0.5 + 0.4 * s(pi * x) * s(pi * y)
        if e == 2:
            return 0.5 + 0.4 * s(pi * x) * s(pi * y) * s(pi * z)
        if e == 3:
            return 0.5 + 0.4 * s(pi * (x - 0.5 * t)) + 0.0 * y
        if e == 4:
            return 0.5 + 0.4 * s(pi * (x - 0.5 * t)) * s(pi * (y - 0.5 * t))
        return 0.5 + 0.4 * s(pi * (x - 0.5 * t)) * s(pi * (y - 0.5 * t)) * s(pi * (z - 0.5 * t))

    def u(self, X, t):
        x, y, z = X
        xp = _xp(x)
        s, c, pi = xp.sin, xp.cos, np.pi
        e = self.example
        zero = 0.0 * x
        if e == 1:
            return [-2.0 * s(pi * x) ** 2 * s(pi * y) * c(pi * y),
                    2.0 * s(pi * y) ** 2 * s(pi * x) * c(pi * x), zero]
        if e == 2:
            return [s(pi * x) ** 2 * s(pi * y) * c(pi * y) * s(pi * z) * c(pi * z),
                    s(pi * y) ** 2 * s(pi * x) * c(pi * x) * s(pi * z) * c(pi * z),
                    -2.0 * s(pi * z) ** 2 * s(pi * x) * c(pi * x) * s(pi * y) * c(pi * y)]
        v = 0.5 + 1.0 / self.eps(X, t)
        if e == 3:
            return [v, zero, zero]
        if e == 4:
            return [v, v, zero]
        return [v, v, v]

    def p(self, X, t):
        x, y, z = X
        s, pi = _xp(x).sin, np.pi
        e = self.example
        if e == 1:
            return s(pi * x) * s(pi * y)
        if e == 2:
            return s(pi * x) * s(pi * y) * s(pi * z)
        if e == 3:
            return s(pi * (x - 0.5 * t)) + 0.0 * y
        if e == 4:
            return s(pi * (x - 0.5 * t)) * s(pi * (y - 0.5 * t))
        return s(pi * (x - 0.5 * t)) * s(pi * (y - 0.5 * t)) * s(pi * (z - 0.5 * t))

    def coords(self):
        nz, ny, nx = self.shape
        x, y, z = _grid(self.shape)
        return (x * self.dx, y * self.dx, z * self.dx)

    def force(self, X, t, rho: float = 1.0):
        """F_MMS of Sec. 3: d_t(phi rho u) + div(phi rho u u) + phi grad p
        - nu div(phi rho (grad u + u grad)), physical units, by central
        finite differences."""
        h = self.h_fd
        d = self.dim
        axes = range(3 if d == 3 else (2 if d == 2 else 1))
        F = []
        for a in range(3):
            if a not in axes:
                F.append(0.0 * X[0])
                continue

            def mom(Y, t, a=a):
                return self.eps(Y, t) * rho * self.u(Y, t)[a]
            term = _d(mom, 3, h)(X, t)
            for b in axes:
                def flux(Y, t, a=a, b=b):
                    uu = self.u(Y, t)
                    return self.eps(Y, t) * rho * uu[a] * uu[b]
                term = term + _d(flux, b, h)(X, t)
            term = term + self.eps(X, t) * _d(self.p, a, h)(X, t)
            for b in axes:
                def visc(Y, t, a=a, b=b):
                    du_ab = _d(lambda Z, s: self.u(Z, s)[a], b, h)(Y, t)
                    du_ba = _d(lambda Z, s: self.u(Z, s)[b], a, h)(Y, t)
                    return self.eps(Y, t) * rho * (du_ab + du_ba)
                term = term - self.nu * _d(visc, b, h)(X, t)
            F.append(term)
        return F

    def force_closed(self, X, t, rho: float = 1.0):
        """Closed form of F_MMS for the travelling-wave Examples 3-5.

        With xi_k = x_k - t/2 on the active axes D, S = prod_k sin(pi xi_k),
        phi = 0.5 + 0.4 S, u_a = 0.5 + 1/phi (a in D) and p = S, the four
        terms of F_MMS reduce to
          F_a = -(1/phi^2) sum_b d_b phi + phi d_a S
                + nu sum_b [(d_bb phi + d_ab phi)/phi - (d_b phi + d_a phi) d_b phi/phi^2]
        (sums over b in D; the time derivative and the convective flux
        combine into the first term)."""
        if self.stationary:
            raise ValueError("closed form only for the transient examples")
        axes = list(range(self.dim))
        pi = np.pi
        xp = _xp(X[0])
        xi = [X[k] - 0.5 * t for k in axes]
        sn = [xp.sin(pi * v) for v in xi]
        cs = [xp.cos(pi * v) for v in xi]

        def prod_except(skip):
            out = 1.0
            for k in axes:
                if k not in skip:
                    out = out * sn[k]
            return out
        S = prod_except(())
        dS = [pi * cs[a] * prod_except((a,)) for a in axes]

        def d2S(a, b):
            if a == b:
                return -pi * pi * S
            return pi * pi * cs[a] * cs[b] * prod_except((a, b))
        eps = 0.5 + 0.4 * S
        de = [0.4 * v for v in dS]
        F = []
        for a in range(3):
            if a not in axes:
                F.append(0.0 * X[0])
                continue
            term = -sum(de) / (eps * eps) + eps * dS[a]
            visc = 0.0
            for b in axes:
                visc = visc + (0.4 * d2S(b, b) + 0.4 * d2S(a, b)) / eps \
                    - (de[b] + de[a]) * de[b] / (eps * eps)
            F.append(term + self.nu * visc)
        return F

    def lattice_series(self, n0: int, nsteps: int):
        """Exact per-step lattice-unit phi and F_MMS for steps n0..n0+nsteps-1:
        arrays of shape (nsteps, N) and (nsteps, 3, N).  Transient examples
        only (the stationary ones do not change in time)."""
        X = self.coords()
        t = (n0 + np.arange(nsteps, dtype=np.float64)) * self.dt
        Xt = [np.broadcast_to(c, (nsteps,) + c.shape) for c in X]
        tt = t.reshape((nsteps, 1, 1, 1))
        eps = self.eps(Xt, tt).reshape(nsteps, -1)
        F = np.stack(self.force_closed(Xt, tt), axis=1).reshape(nsteps, 3, -1)
        return np.ascontiguousarray(eps), np.ascontiguousarray(F * self.dt * self.dt / self.dx)

    def lattice_series_torch(self, n0: int, nsteps: int, device="cuda", dtype=None):
        """lattice_series evaluated with torch on `device`: the exact per-step
        phi (nsteps, N) and F_MMS (nsteps, 3, N) of a transient example,
        generated where the solver reads them."""
        import torch
        dtype = dtype or torch.float64
        X = [torch.as_tensor(c, dtype=torch.float64, device=device) for c in self.coords()]
        t = (n0 + torch.arange(nsteps, dtype=torch.float64, device=device)) * self.dt
        Xt = [c.unsqueeze(0).expand((nsteps,) + tuple(c.shape)) for c in X]
        tt = t.reshape(nsteps, 1, 1, 1)
        eps = self.eps(Xt, tt).reshape(nsteps, -1)
        F = torch.stack([f.expand((nsteps,) + tuple(X[0].shape)) if torch.is_tensor(f) else f
                         for f in self.force_closed(Xt, tt)], dim=1).reshape(nsteps, 3, -1)
        F = F * (self.dt * self.dt / self.dx)
        return eps.to(dtype).contiguous(), F.to(dtype).contiguous()

    # lattice-unit views at time step n
    def lattice_fields(self, n: int):
        """dict(eps, deps_dt, force, dforce_dt, u, p) in lattice units at step n
        (the force by finite differences for Examples 1-2, in closed form for
        Examples 3-5).

        Force density: F_L = F dt^2 / dx; velocity u_L = u dt/dx; pressure
        p_L = p dt^2/dx^2; time derivatives are per time step."""
        X = self.coords()
        t = n * self.dt
        dx, dt = self.dx, self.dt
        eps = self.eps(X, t)
        deps = _d(self.eps, 3, self.h_fd * 1e-2)(X, t) * dt
        force = self.force if self.stationary else self.force_closed
        F = np.stack(force(X, t)) * dt * dt / dx
        dF = None
        if not self.stationary:
            dF = np.stack(_d(lambda Y, s: np.stack(force(Y, s)), 3, 1e-4)(X, t)) * dt * dt / dx * dt
        u = np.stack(self.u(X, t)) * dt / dx
        p = self.p(X, t) * dt * dt / (dx * dx)
        return {"eps": eps, "deps_dt": deps if not self.stationary else None,
                "force": F, "dforce_dt": dF, "u": u, "p": p}

    def steps_for(self, t_end: float) -> int:
        return int(round(t_end / self.dt))


def error_norms(q: np.ndarray, q_ref: np.ndarray) -> dict:
    """L1, L2 and Linf norms over nodal values (Sec. 3 error definitions);
    vector fields: |.| is the Euclidean norm over the leading axis."""
    diff = np.asarray(q, dtype=np.float64) - np.asarray(q_ref, dtype=np.float64)
    if diff.ndim == 4:
        mag = np.sqrt((diff ** 2).sum(axis=0))
    else:
        mag = np.abs(diff)
    n = mag.size
    return {"L1": float(mag.sum() / n), "L2": float(math.sqrt((mag ** 2).sum() / n)),
            "Linf": float(mag.max())}


# --------------------------------------------------------------------------
# Batched and served workloads
# --------------------------------------------------------------------------

@dataclass
class LatticeSpec:
    """One independent lattice problem of a batch or a served request."""
    lattice: str
    shape: tuple           # (nz, ny, nx)
    tau: float
    amp: float
    seed: int
    kind: str = "sine"     # "sine" or "spheres"
    steps: int = 1000
    residual_tol: float = 0.0
    g: tuple = (1e-6, 0.0, 0.0)

    @property
    def cells(self) -> int:
        return int(np.prod(self.shape))

    def eps(self) -> np.ndarray:
        if self.kind == "spheres":
            r = max(2.0, self.shape[-1] / 32.0)
            return eps_random_spheres(self.shape, seed_offset=self.seed, rmin=r,
                                      rmax=3 * r, sigma=max(1.0, 0.75 * r), wall_axis=None)
        return eps_product_sine(self.shape, self.amp)


def batch_specs(count: int = 256, seed_offset: int = 4000, d2_sides=(32, 512),
                d3_sides=(32, 128), steps: int = 1000) -> list:
    """Half D2Q9 squares (side uniform in d2_sides), half D3Q19 cubes (side
    uniform in d3_sides), periodic; amplitude U[0.05, 0.3]; tau U[0.55, 1.2]."""
    g = rng(seed_offset)
    out = []
    for j in range(count):
        if j < count // 2:
            s = int(g.integers(d2_sides[0], d2_sides[1] + 1))
            shape, lat = (1, s, s), "D2Q9"
        else:
            s = int(g.integers(d3_sides[0], d3_sides[1] + 1))
            shape, lat = (s, s, s), "D3Q19"
        out.append(LatticeSpec(lat, shape, float(g.uniform(0.55, 1.2)),
                               float(g.uniform(0.05, 0.3)), seed_offset + j, steps=steps))
    return out


def poisson_requests(rate: float, count: int, seed_offset: int = 5000,
                     sides=(32, 192), steps=(500, 20000), residual_share: float = 0.5,
                     sphere_share: float = 0.5) -> list:
    """Arrival trace of D3Q19 solve requests: exponential inter-arrival times
    of mean 1/rate seconds; side log-uniform in ``sides``; phi from random
    spheres or a product sine (50/50); a step budget log-uniform in ``steps``,
    or (half of them) a steady-state residual target of 1e-8 with that budget
    as the cap.  Returns [(arrival_s, LatticeSpec)]."""
    g = rng(seed_offset)
    # arrival times from a stream of their own: the same seed gives the same
    # sequence of problems at every rate
    g_arrival = rng(seed_offset + 1_000_003)
    t = 0.0
    out = []
    for j in range(count):
        t += float(g_arrival.exponential(1.0 / rate))
        side = int(round(math.exp(g.uniform(math.log(sides[0]), math.log(sides[1])))))
        nsteps = int(round(math.exp(g.uniform(math.log(steps[0]), math.log(steps[1])))))
        kind = "spheres" if g.uniform() < sphere_share else "sine"
        tol = 1e-8 if g.uniform() < residual_share else 0.0
        spec = LatticeSpec("D3Q19", (side, side, side), float(g.uniform(0.55, 1.2)),
                           float(g.uniform(0.05, 0.3)), seed_offset + j, kind=kind,
                           steps=nsteps, residual_tol=tol)
        out.append((t, spec))
    return out


_EPS_CACHE = {}


def cached_eps(spec) -> np.ndarray:
    """spec.eps() as float32, kept for reuse (the same problem served at
    several arrival rates is generated once)."""
    key = (spec.kind, spec.shape, spec.amp, spec.seed)
    if key not in _EPS_CACHE:
        _EPS_CACHE[key] = spec.eps().astype(np.float32).ravel()
    return _EPS_CACHE[key]
