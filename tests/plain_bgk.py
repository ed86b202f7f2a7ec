"""A plain BGK lattice Boltzmann solver with Guo forcing, written in numpy,
independently of the oracle.

It is what the consistent VANSE scheme must reduce to when the volume
fraction is one everywhere (Sec. 2.2: then int phi dV = 1, grad phi = 0,
F_PC = 0 and rho~ = sum f).  It builds its velocity sets from the group
weights alone (sorted by |xi|^2, not by the oracle's table order), streams
with ``np.roll`` and treats walls with masks, so it shares neither layout nor
loop structure with the oracle.  Results are compared through the
macroscopic fields only.
"""
from __future__ import annotations

import itertools

import numpy as np

GROUP_WEIGHTS = {
    "D1Q3": (1, {0: 2 / 3, 1: 1 / 6}),
    "D2Q9": (2, {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}),
    "D3Q19": (3, {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}),
    "D3Q27": (3, {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}),
}


def velocity_set(name):
    d, gw = GROUP_WEIGHTS[name]
    c = [v for v in itertools.product((-1, 0, 1), repeat=d) if sum(x * x for x in v) in gw]
    c.sort(key=lambda v: (sum(x * x for x in v), v))
    c = np.array(c, dtype=np.int64)
    w = np.array([gw[int((v * v).sum())] for v in c])
    return c, w


class PlainBGK:
    """f has shape (Q,) + lattice shape with axes ordered (x, y[, z])."""

    def __init__(self, name, shape_xyz, tau, g, wall_axis=None):
        self.c, self.w = velocity_set(name)
        self.d = self.c.shape[1]
        self.shape = tuple(shape_xyz)
        self.tau = tau
        self.g = np.asarray(g[: self.d], dtype=np.float64)
        self.solid = np.zeros(self.shape, dtype=bool)
        if wall_axis is not None:
            idx = [slice(None)] * self.d
            idx[wall_axis] = 0
            self.solid[tuple(idx)] = True
            idx[wall_axis] = -1
            self.solid[tuple(idx)] = True
        self.opp = np.array([int(np.where((self.c == -v).all(axis=1))[0][0]) for v in self.c])

    def equilibrium(self, rho, u):
        cu = np.tensordot(self.c.astype(np.float64), u, axes=(1, 0))
        usq = (u * u).sum(axis=0)
        return self.w.reshape((-1,) + (1,) * self.d) * rho * (
            1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * usq)

    def macro(self, f):
        rho = f.sum(axis=0)
        j = np.tensordot(self.c.T.astype(np.float64), f, axes=(1, 0))
        F = np.broadcast_to(self.g.reshape((-1,) + (1,) * self.d), j.shape)
        u = (j + 0.5 * F) / np.where(self.solid, 1.0, rho)
        return rho, u, F

    def step(self, f):
        rho, u, F = self.macro(f)
        feq = self.equilibrium(rho, u)
        # Guo et al. (2002): (1 - 1/(2 tau)) w_i [(c - u)/cs^2 + (c.u) c/cs^4] . F
        cF = np.tensordot(self.c.astype(np.float64), F, axes=(1, 0))
        cu = np.tensordot(self.c.astype(np.float64), u, axes=(1, 0))
        uF = (u * F).sum(axis=0)
        src = (1 - 0.5 / self.tau) * self.w.reshape((-1,) + (1,) * self.d) * (
            3 * (cF - uF) + 9 * cu * cF)
        post = f - (f - feq) / self.tau + src
        post[:, self.solid] = 0.0
        new = np.empty_like(f)
        for i, v in enumerate(self.c):
            new[i] = np.roll(post[i], shift=tuple(int(s) for s in v), axis=tuple(range(self.d)))
        # halfway bounce-back: what streamed into a solid cell returns reversed
        for i, v in enumerate(self.c):
            hit = new[i] * self.solid
            back = np.roll(hit, shift=tuple(-int(s) for s in v), axis=tuple(range(self.d)))
            new[self.opp[i]] += back
        new[:, self.solid] = 0.0
        return new
