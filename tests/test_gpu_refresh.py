"""Refreshes of phi (Sec. 2.2: phi(x, t) varies in space and time; the
caller refreshes phi_ref and d_t phi, and phi at step n is
phi_ref + (n - n_ref) d_t phi).

- A refresh staged on the library's copy stream before the steps it
  overlaps and committed after them leaves the lattice bit-identical to the
  same refresh given to set_epsilon at the commit (host and device sources,
  FP32 and FP16 storage, rows padded to the pitch).
- A rejected refresh, by either route, leaves the lattice as it was: it then
  advances bit-identically to a lattice that never saw the refresh (a
  rejected d_t phi must not reach the field the steps read).
- The call-order rules of the header (LBM_ESTATE) hold."""
import numpy as np
import pytest

from paper_2208_09267_gb300 import inputs as I
from paper_2208_09267_gb300 import lbm

pytestmark = pytest.mark.gpu

K = 10  # steps between refreshes
EINVAL, ESTATE = -1, -6


def _fields(shape, n):
    """phi_ref and d_t phi of the refresh at step n (a travelling wave)."""
    nz, ny, nx = shape
    e, d = I.eps_travelling_wave(nx, float(n), T=200.0, shape=shape)
    return e.ravel().astype(np.float32), d.ravel().astype(np.float32)


def _lattice(shape, storage="fp32"):
    nz, ny, nx = shape
    lat = lbm.Lattice("D3Q19", (nx, ny, nz), tau=0.6, storage=storage)
    e, d = _fields(shape, 0)
    lat.set_epsilon(e, d, 0)
    lat.set_force((1e-5, 0.0, 0.0))
    lat.init_equilibrium()
    return lat


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("source", ["host", "device"])
def test_staged_refresh_equals_set_epsilon(storage, source):
    import torch
    shape = (12, 20, 45)  # nx = 45: rows stored at a pitch of 48
    a, b = _lattice(shape, storage), _lattice(shape, storage)
    if source == "device":
        conv = lambda x: torch.as_tensor(x).cuda()  # noqa: E731
    else:
        conv = lambda x: x  # noqa: E731
    for j in range(1, 6):
        e, d = _fields(shape, j * K)
        ea, da, eb, db = conv(e), conv(d), conv(e), conv(d)
        b.stage_epsilon(eb, db, j * K)
        a.step(K, check_every=-1)
        b.step(K, check_every=-1)
        a.set_epsilon(ea, da, j * K)
        b.commit_epsilon()
    # a static refresh (no d_t phi) by both routes
    e, _ = _fields(shape, 6 * K)
    b.stage_epsilon(conv(e), None, 6 * K)
    a.step(K, check_every=-1)
    b.step(K, check_every=-1)
    a.set_epsilon(conv(e), None, 6 * K)
    b.commit_epsilon()
    sa, sb = a.step(K), b.step(K)
    assert sa["steps_done"] == sb["steps_done"] == 7 * K
    assert np.array_equal(a.populations(), b.populations())
    ma, mb = a.moments(), b.moments()
    assert np.array_equal(ma["p"], mb["p"]) and np.array_equal(ma["u"], mb["u"])
    a.close()
    b.close()


@pytest.mark.parametrize("route,field", [("set", "deps"), ("stage", "deps"), ("stage", "eps")])
def test_rejected_refresh_leaves_the_lattice_unchanged(route, field):
    shape = (8, 10, 24)
    a, ref = _lattice(shape), _lattice(shape)
    a.step(K, check_every=-1)
    ref.step(K, check_every=-1)
    e, d = _fields(shape, K)
    if field == "deps":
        d = d.copy()
        d[123] = np.nan
        where = "deps_dt[123]"
    else:
        e = e.copy()
        e[77] = 0.0
        where = "eps_ref[77]"
    with pytest.raises(lbm.LbmError) as ex:
        if route == "set":
            a.set_epsilon(e, d, K)
        else:
            a.stage_epsilon(e, d, K)
            a.commit_epsilon()
    assert ex.value.code == EINVAL and where in str(ex.value)
    sa, sr = a.step(2 * K), ref.step(2 * K)
    assert not sa["nan_seen"]
    assert np.array_equal(a.populations(), ref.populations())
    # the handle still takes refreshes by both routes afterwards
    e, d = _fields(shape, 3 * K)
    a.stage_epsilon(e, d, 3 * K)
    a.commit_epsilon()
    ref.set_epsilon(e, d, 3 * K)
    a.step(K)
    ref.step(K)
    assert np.array_equal(a.populations(), ref.populations())
    a.close()
    ref.close()


def test_staged_refresh_call_order():
    shape = (4, 6, 16)
    a = _lattice(shape)
    state = a.save_state()
    e, d = _fields(shape, K)
    with pytest.raises(lbm.LbmError) as ex:
        a.commit_epsilon()            # nothing staged
    assert ex.value.code == ESTATE
    a.stage_epsilon(e, d, K)
    for call in (lambda: a.stage_epsilon(e, d, K), lambda: a.set_epsilon(e, d, K),
                 lambda: a.load_state(state)):
        with pytest.raises(lbm.LbmError) as ex:
            call()
        assert ex.value.code == ESTATE
    a.step(3)                         # steps run on the current phi meanwhile
    a.commit_epsilon()
    a.step(3)
    a.load_state(state)               # allowed again after the commit
    a.close()
    f64 = lbm.Lattice("D3Q19", (16, 6, 4), tau=0.6, storage="fp64")
    with pytest.raises(lbm.LbmError) as ex:
        f64.stage_epsilon(e, d, K)
    assert ex.value.code == EINVAL
    f64.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_switching_between_static_and_varying_phi(storage):
    """A lattice whose row kernel stages fewer, larger stages when phi has a
    time derivative (D3Q27 rows of 320 cells: 2 stages, 3 without d_t phi)
    steps through graph replays with static phi, then with a varying phi,
    then static again: each phase takes the stage layout of its phi, and the
    run equals the one-cell-per-thread kernel's (populations to float
    rounding in FP32; the moments within the FP16 bar in FP16)."""
    shape = (320, 5, 6)
    nx, ny, nz = shape
    rng = np.random.default_rng(5)
    e0 = (0.6 + 0.3 * rng.random(nx * ny * nz)).astype(np.float32)
    d1 = (1e-4 * rng.standard_normal(nx * ny * nz)).astype(np.float32)
    lats = []
    for kern in ("row", "cell"):
        lat = lbm.Lattice("D3Q27", shape, tau=0.6, storage=storage, walls=4, kernel=kern, tuned=False)
        assert lat.row_kernel == (kern == "row")
        lat.set_epsilon(e0)
        lat.set_force((1e-5, 0.0, 0.0))
        lat.init_equilibrium()
        lat.step(130, check_every=-1)             # graph replays, static phi
        lat.set_epsilon(e0, d1, 130)
        lat.step(130, check_every=-1)             # varying phi
        lat.set_epsilon(np.clip(e0 + 130 * d1, 0.05, 1.0))
        st = lat.step(131)                        # static again, ends with a check step
        assert not st["nan_seen"]
        lats.append(lat)
    row, cell = lats
    if storage == "fp32":
        pr, pc = row.populations(), cell.populations()
        assert np.abs(pr - pc).max() <= 4e-6 * np.abs(pc).max()
    else:
        mr, mc = row.moments(), cell.moments()
        ur, uc = mr["u"].ravel(), mc["u"].ravel()
        assert np.linalg.norm(ur - uc) <= 2e-3 * np.linalg.norm(uc)
