"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test pins one part of the oracle to something other than the oracle
itself: the tables the paper prints (tests/golden), moment identities of the
equilibrium and forcing (Sec. 2.2 eqs. (M0)-(M3), Appendix A eqs. (M0F)-(M2F)),
an independently written plain BGK solver for the phi == 1 reduction,
exact invariants (mass, momentum, homogeneity) and closed-form flows.
"""
from fractions import Fraction
import itertools

import numpy as np
import pytest

import oracle
from conftest import golden
from plain_bgk import PlainBGK

CS2 = 1.0 / 3.0
LATS = ["D2Q9", "D3Q19", "D3Q27", "D1Q3"]


def _read_table(name):
    rows = []
    with open(golden(name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- tables

@pytest.mark.parametrize("lat", LATS)
def test_lattice_weights_match_printed_tables(lat):
    """Tables "latt_par" and "latt_3d" (D3Q19: textbook weights)."""
    c, w, opp = oracle.velocity_set(oracle.LATTICES[lat])
    expect = {int(r[1]): (int(r[2]), float(Fraction(r[3])))
              for r in _read_table("lattice_weights.txt") if r[0] == lat}
    norms = (c * c).sum(axis=1)
    assert norms[0] == 0 and c.shape[0] == sum(v[0] for v in expect.values())
    for k, (count, weight) in expect.items():
        sel = norms == k
        assert sel.sum() == count
        assert np.all(w[sel] == weight)
    # every direction appears once and its opposite is recorded
    assert len({tuple(v) for v in c}) == c.shape[0]
    assert np.all(c[opp] == -c)


@pytest.mark.parametrize("lat", LATS)
def test_lattice_isotropy(lat):
    """sum w = 1, sum w xi = 0, sum w xi xi = cs2 I, fourth-order isotropy
    sum w xi_a xi_b xi_c xi_d = cs2^2 (d_ab d_cd + d_ac d_bd + d_ad d_bc)."""
    c, w, _ = oracle.velocity_set(oracle.LATTICES[lat])
    d = oracle.DIM_OF[oracle.LATTICES[lat]]
    c = c[:, :d].astype(float)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ c).max() < 1e-16
    assert np.abs(np.einsum("i,ia,ib->ab", w, c, c) - CS2 * np.eye(d)).max() < 1e-15
    T4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    I = np.eye(d)
    ref = CS2 ** 2 * (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
                      + np.einsum("ad,bc->abcd", I, I))
    assert np.abs(T4 - ref).max() < 1e-15


def test_quadrature_weights_match_table():
    """Table "weights"; each row sums to one over the 2d+1 points."""
    for d, w0, w1 in _read_table("quadrature_weights.txt"):
        d = int(d)
        got = oracle.quad_weights(d)
        assert got[0] == float(Fraction(w0)) and got[1] == float(Fraction(w1))
        assert abs(got[0] + 2 * d * got[1] - 1.0) < 1e-15
    with pytest.raises(ValueError):
        oracle.quad_weights(4)


@pytest.mark.parametrize("quad_dim,axes", [(1, 1), (1, 2), (2, 3), (3, 7)])
def test_quadrature_equals_laplacian_form(quad_dim, axes):
    """eq. (quad) rearranged, eq. (latDiffRuleIIre): the quadrature equals
    phi + varpi_{i!=0} lap_h phi, with the discrete Laplacian over the
    quadrature axes.  The oracle's int phi dV is recovered as M0 / rho~."""
    lat = "D3Q19" if axes == 7 else "D2Q9"
    shape = (5, 6, 7) if lat == "D3Q19" else (1, 6, 7)
    rng = np.random.default_rng(1)
    eps = 0.5 + 0.4 * rng.random(shape)
    P = oracle.Problem(lat, shape[2], shape[1], shape[0], quad_dim=quad_dim,
                       quad_axes=axes, eps_ref=eps)
    f = P.init()
    m = P.moments(f, 0)
    integral = m["M0"] / m["rho"]
    w1 = oracle.quad_weights(quad_dim)[1]
    lap = np.zeros(shape)
    for a in range(3):
        if axes & (1 << a):
            ax = 2 - a
            lap += np.roll(eps, 1, ax) + np.roll(eps, -1, ax) - 2 * eps
    assert np.abs(integral - (eps + w1 * lap)).max() < 1e-14


# ------------------------------------------------------ moment identities

def _random_cell(rng, d):
    M0 = 0.3 + rng.random()
    u = np.zeros(3)
    F = np.zeros(3)
    u[:d] = 0.1 * (rng.random(d) - 0.5)
    F[:d] = 1e-2 * (rng.random(d) - 0.5)
    return M0, u, F


@pytest.mark.parametrize("lat", LATS)
def test_equilibrium_moments(lat):
    """Sec. 2.2 eqs. (M0)-(M3): with the integral mass M0 = rho~ int phi,
    sum f^eq = M0, sum xi f^eq = M0 u, sum xi xi f^eq = M0 uu + cs2 M0 I,
    and (eq. (M3), printed garbled; standard form) sum xi xi xi f^eq =
    cs2 M0 (u_a d_bc + u_b d_ac + u_c d_ab)."""
    rng = np.random.default_rng(2)
    c, w, _ = oracle.velocity_set(oracle.LATTICES[lat])
    d = oracle.DIM_OF[oracle.LATTICES[lat]]
    c = c[:, :d].astype(float)
    I = np.eye(d)
    for _ in range(20):
        M0, u, F = _random_cell(rng, d)
        feq, _ = oracle.cell_terms(oracle.LATTICES[lat], M0, u, F, 0.7)
        ud = u[:d]
        assert abs(feq.sum() - M0) < 1e-14 * M0
        assert np.abs(c.T @ feq - M0 * ud).max() < 1e-15
        M2 = np.einsum("i,ia,ib->ab", feq, c, c)
        assert np.abs(M2 - (M0 * np.outer(ud, ud) + CS2 * M0 * I)).max() < 1e-14
        M3 = np.einsum("i,ia,ib,ic->abc", feq, c, c, c)
        ref = CS2 * M0 * (np.einsum("a,bc->abc", ud, I) + np.einsum("b,ac->abc", ud, I)
                          + np.einsum("c,ab->abc", ud, I))
        assert np.abs(M3 - ref).max() < 1e-15


@pytest.mark.parametrize("lat", LATS)
def test_forcing_moments(lat):
    """Appendix A eqs. (M0F)-(M2F): sum Omega^F = 0, sum xi Omega^F =
    (1 - 1/(2 tau)) F, sum xi xi Omega^F = (1 - 1/(2 tau)) (F u + u F)."""
    rng = np.random.default_rng(3)
    c, w, _ = oracle.velocity_set(oracle.LATTICES[lat])
    d = oracle.DIM_OF[oracle.LATTICES[lat]]
    c = c[:, :d].astype(float)
    for tau in (0.51, 0.8, 1.7):
        M0, u, F = _random_cell(rng, d)
        _, om = oracle.cell_terms(oracle.LATTICES[lat], M0, u, F, tau)
        k = 1 - 0.5 / tau
        assert abs(om.sum()) < 1e-18
        assert np.abs(c.T @ om - k * F[:d]).max() < 1e-18
        M2F = np.einsum("i,ia,ib->ab", om, c, c)
        assert np.abs(M2F - k * (np.outer(F[:d], u[:d]) + np.outer(u[:d], F[:d]))).max() < 1e-18


@pytest.mark.parametrize("lat", LATS)
def test_cell_terms_against_printed_tensor_forms(lat):
    """Direct evaluation of eq. (equilibrium)/(feq) and of the Guo term in
    the tensor notation of Sec. 2.2 (c_s^2 = 1/3 as a float, loops over
    alpha, beta) agrees with the oracle's expanded constants."""
    rng = np.random.default_rng(4)
    c, w, _ = oracle.velocity_set(oracle.LATTICES[lat])
    d = oracle.DIM_OF[oracle.LATTICES[lat]]
    for _ in range(5):
        M0, u, F = _random_cell(rng, d)
        tau = 0.5 + rng.random()
        feq, om = oracle.cell_terms(oracle.LATTICES[lat], M0, u, F, tau)
        for i in range(len(w)):
            xi = c[i, :d].astype(float)
            t1 = sum(xi[a] * u[a] for a in range(d)) / CS2
            t2 = sum((xi[a] * xi[b] - CS2 * (a == b)) * u[a] * u[b]
                     for a in range(d) for b in range(d)) / (2 * CS2 ** 2)
            assert abs(w[i] * M0 * (1 + t1 + t2) - feq[i]) < 1e-15
            g = sum((xi[a] / CS2 + sum((xi[a] * xi[b] - CS2 * (a == b)) * u[b]
                                       for b in range(d)) / CS2 ** 2) * F[a] for a in range(d))
            assert abs((1 - 1 / (2 * tau)) * w[i] * g - om[i]) < 1e-17


# --------------------------------------------- the phi == 1 reduction

def _to_xyz(a, d):
    a = np.asarray(a)
    return a[0, 0] if d == 1 else (a[0].T if d == 2 else a.T)


def _dim(lat):
    return oracle.DIM_OF[oracle.LATTICES[lat]]


def _shape(d, two, three, one=(1, 1, 12)):
    """(nz, ny, nx) of a test lattice of dimension d."""
    return one if d == 1 else (two if d == 2 else three)


def _wall_bits(d, walls):
    """y walls, or x walls on a one-dimensional lattice."""
    return (1 if d == 1 else 2) if walls else 0


@pytest.mark.parametrize("lat", LATS)
@pytest.mark.parametrize("walls", [0, 2])
def test_unit_volume_fraction_reduces_to_plain_bgk(lat, walls):
    """phi == 1: int phi = 1, grad phi = 0, F_PC = 0 and rho~ = sum f, so the
    scheme is plain BGK with Guo forcing (and halfway bounce-back at walls)."""
    d = _dim(lat)
    shape = _shape(d, (1, 9, 7), (5, 8, 6), (1, 1, 11))
    rng = np.random.default_rng(5)
    p0 = 1e-3 * rng.standard_normal(shape)
    u0 = 1e-2 * rng.standard_normal((d,) + shape)
    g = (2e-5, -1e-5, 3e-6)
    tau = 0.62
    P = oracle.Problem(lat, shape[2], shape[1], shape[0], tau=tau, g=g, walls=_wall_bits(d, walls))
    f = P.init(p0=p0, u0=u0)
    ref = PlainBGK(lat, shape[::-1][:d], tau, g,
                   wall_axis=(0 if d == 1 else 1) if walls else None)
    rho0 = _to_xyz(1 + 3 * p0, d)
    uu = np.stack([_to_xyz(u0[a], d) for a in range(d)])
    fr = ref.equilibrium(rho0, uu)
    fr[:, ref.solid] = 0
    steps = 25
    f = P.run(f, 0, steps)
    for _ in range(steps):
        fr = ref.step(fr)
    m = P.moments(f, steps)
    rho_r, u_r, _ = ref.macro(fr)
    fluid = ~ref.solid
    assert np.abs(_to_xyz(m["M0"], d)[fluid] - rho_r[fluid]).max() < 1e-14
    for a in range(d):
        ua = _to_xyz(m["u"][a], d)
        assert np.abs(ua[fluid] - u_r[a][fluid]).max() < 1e-15


@pytest.mark.parametrize("lat", LATS)
def test_homogeneity_in_constant_volume_fraction(lat):
    """feq and Omega^F are homogeneous of degree one in (M0, F): the run with
    phi == c and force c g equals c times the run with phi == 1 and g."""
    d = _dim(lat)
    shape = _shape(d, (1, 8, 8), (4, 5, 6))
    rng = np.random.default_rng(6)
    u0 = 1e-2 * rng.standard_normal((d,) + shape)
    cst = 0.37
    g = np.array([1e-5, 2e-5, -1e-5])
    P1 = oracle.Problem(lat, shape[2], shape[1], shape[0], tau=0.7, g=g)
    Pc = oracle.Problem(lat, shape[2], shape[1], shape[0], tau=0.7, g=cst * g,
                        eps_ref=np.full(shape, cst))
    f1 = P1.run(P1.init(u0=u0), 0, 30)
    fc = Pc.run(Pc.init(u0=u0), 0, 30)
    assert np.abs(fc - cst * f1).max() < 1e-13 * np.abs(f1).max()


# ------------------------------------------------------------ invariants

def _varying_problem(lat, walls, time_varying=True):
    d = _dim(lat)
    shape = _shape(d, (1, 12, 10), (6, 8, 7), (1, 1, 16))
    walls = _wall_bits(d, walls)
    rng = np.random.default_rng(7)
    eps = 0.55 + 0.3 * rng.random(shape)
    deps = 1e-4 * rng.standard_normal(shape) if time_varying else None
    force = 1e-5 * rng.standard_normal((3,) + shape)
    P = oracle.Problem(lat, shape[2], shape[1], shape[0], tau=0.66, g=(1e-5, 0, 0),
                       walls=walls, eps_ref=eps, deps_dt=deps, n_eps=3, force=force)
    return P, shape


@pytest.mark.parametrize("lat", LATS)
@pytest.mark.parametrize("walls", [0, 2])
def test_mass_is_conserved(lat, walls):
    """sum Omega^F = 0 (eq. (M0F)) and sum f^eq = M0: streaming and
    bounce-back move mass, collision keeps it."""
    P, _ = _varying_problem(lat, walls)
    f = P.init(half_force=True, with_integral=True)
    m0 = f.sum()
    for n in range(40):
        f = P.step(f, n)
        assert abs(f.sum() - m0) < 1e-13 * m0


@pytest.mark.parametrize("lat", LATS)
def test_momentum_balance(lat):
    """Periodic lattice: sum_x J(n+1) - sum_x J(n) = sum_x F(n), the Guo
    momentum input (first moment of the update with eq. (velocity))."""
    P, shape = _varying_problem(lat, 0)
    c, _, _ = oracle.velocity_set(P.lattice)
    f = P.init(half_force=True, with_integral=True)
    for n in range(10):
        J0 = f @ c.astype(float)
        F = P.forces(f, n).reshape(3, -1).T
        f1 = P.step(f, n)
        J1 = f1 @ c.astype(float)
        assert np.abs(J1.sum(0) - J0.sum(0) - F.sum(0)).max() < 1e-13 * np.abs(F).sum()
        f = f1


@pytest.mark.parametrize("lat", LATS)
def test_half_force_init_reports_initial_state(lat):
    """With the half-force shift the velocity of eq. (velocity) at t = 0 is
    u0, and with the integral mass the pressure is p0."""
    P, shape = _varying_problem(lat, 0, time_varying=False)
    d = P.d
    rng = np.random.default_rng(8)
    u0 = 1e-2 * rng.standard_normal((d,) + shape)
    p0 = 1e-3 * rng.standard_normal(shape)
    m = P.moments(P.init(p0=p0, u0=u0, half_force=True, with_integral=True), 0)
    assert np.abs(m["u"][:d] - u0).max() < 1e-16
    assert np.abs(m["p"] - p0).max() < 1e-15


def test_time_extrapolation_matches_exact_series():
    """phi_n = phi_ref + (n - n_ref) d_t phi and F_n likewise: a run with the
    pair equals, bit for bit, a run fed the extrapolated fields step by step."""
    P, shape = _varying_problem("D3Q19", 2)
    N = P.n
    dF = 1e-7 * np.random.default_rng(9).standard_normal(3 * N)
    P.set_force(P.g, P.force, dF, 2)
    f0 = P.init(with_integral=True)
    steps = 12
    fa = P.run(f0, 5, steps)
    es = np.stack([(P.eps_ref + (n - P.n_eps) * P.deps_dt).ravel() for n in range(5, 5 + steps)])
    fs = np.stack([P.force.ravel() + (n - P.n_force) * dF for n in range(5, 5 + steps)])
    fb = P.run_series(f0, 5, es, fs)
    assert np.array_equal(fa, fb)


# --------------------------------------------------------- closed forms

@pytest.mark.parametrize("lat", LATS[:3])
def test_poiseuille_exact_at_magic_tau(lat):
    """phi == 1 channel between halfway bounce-back walls: BGK with Guo
    forcing reproduces the parabola u = g/(2 nu) (y - y0)(y1 - y) exactly
    when tau = 1/2 + sqrt(3/16) (walls at y0 = 1/2, y1 = ny - 3/2)."""
    ny = 14
    tau = 0.5 + np.sqrt(3 / 16)
    g = 1e-6
    P = oracle.Problem(lat, 1, ny, 1, tau=tau, walls=2, g=(g, 0, 0), quad_axes=2, quad_dim=1)
    f = P.run(P.init(), 0, 5000)
    u = P.moments(f, 5000)["u"][0][0, :, 0]
    nu = (tau - 0.5) / 3
    y = np.arange(ny)
    ua = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    assert np.abs(u[1:-1] - ua[1:-1]).max() < 1e-9 * ua.max()
    assert u[0] == 0 and u[-1] == 0


def _vanse_channel_error(H, lattice="D2Q9"):
    from scipy.integrate import quad
    ny = H + 2
    tau = 0.8
    nu = (tau - 0.5) / 3
    yw1, yw2 = 0.5, ny - 1.5

    def eps_f(s):
        return 0.75 + 0.2 * np.cos(2 * np.pi * (s - yw1) / H)
    y = np.arange(ny, dtype=float)
    eps = eps_f(y)
    eps[0], eps[-1] = eps[1], eps[-2]
    g = 8 * nu * 1e-3 / H ** 2
    yc = (quad(lambda s: s / eps_f(s), yw1, yw2, epsabs=1e-13)[0]
          / quad(lambda s: 1 / eps_f(s), yw1, yw2, epsabs=1e-13)[0])
    ua = np.array([g / nu * quad(lambda s: (yc - s) / eps_f(s), yw1, v, epsabs=1e-15)[0]
                   for v in y])
    P = oracle.Problem(lattice, 1, ny, 1, tau=tau, walls=2, g=(g, 0, 0), quad_axes=2,
                       quad_dim=1, eps_ref=eps.reshape(1, ny, 1))
    steps = int(8 * H * H / nu)
    f = P.run(P.init(with_integral=True), 0, steps)
    u = P.moments(f, steps)["u"][0][0, :, 0]
    return np.sqrt(np.mean((u[1:-1] - ua[1:-1]) ** 2) / np.mean(ua[1:-1] ** 2))


@pytest.mark.parametrize("lattice", ["D2Q9", "D3Q27"])
def test_vanse_channel_converges_second_order(lattice):
    """Steady channel with phi = phi(y) between walls: eq. (vansEquMom) with
    constant pressure gives nu (phi rho u')' = -g, u = (g/nu) int (y_c - s)
    / phi(s) ds.  The scheme converges to it at second order."""
    e1 = _vanse_channel_error(16, lattice)
    e2 = _vanse_channel_error(32, lattice)
    assert abs(np.log2(e1 / e2) - 2.0) < 0.1
