"""lbm_vanse_moments_noalloc: host read-back of rho, p, u staged in the
library's fixed device array instead of a temporary allocation.  The file is
collected last, so the entry point also runs after every other test has used
the library in the same process; it must pass alone in a fresh process too."""
import ctypes

import numpy as np
import pytest

from paper_2208_09267_gb300 import inputs as I
from paper_2208_09267_gb300 import lbm

pytestmark = pytest.mark.gpu


def _noalloc(lat):
    """Call the entry point through the C ABI with host numpy buffers."""
    rho = np.full(lat.n, np.nan, np.float32)
    p = np.full(lat.n, np.nan, np.float32)
    u = np.full(3 * lat.n, np.nan, np.float32)
    rc = lbm.lib().lbm_vanse_moments_noalloc(lat.handle, rho.ctypes.data, p.ctypes.data,
                                             u.ctypes.data)
    assert rc == 0, lbm.last_error()
    return {"rho": rho, "p": p, "u": u.reshape(3, lat.n)}


def _same(a, b):
    # same kernel, same values: the tolerance is zero
    for k in ("rho", "p", "u"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("lattice,shape,storage,walls", [
    ("D3Q19", (40, 36, 34), "fp32", 0), ("D2Q9", (77, 30, 1), "fp16", 2),
    ("D3Q27", (13, 8, 7), "fp64", 6)])
def test_noalloc_moments_match_moments_on_consecutive_calls(lattice, shape, storage, walls):
    nx, ny, nz = shape
    lat = lbm.Lattice(lattice, shape, tau=0.6, storage=storage, walls=walls)
    rng = np.random.default_rng(I.MASTER_SEED + 77)
    lat.set_epsilon((0.6 + 0.35 * rng.random(nx * ny * nz)).astype(np.float32))
    lat.set_force((2e-5, 1e-6, 0.0))
    lat.init_equilibrium(integral=True, half_force=True)
    lat.step(21)
    first = _noalloc(lat)
    second = _noalloc(lat)   # two calls in a row share the staging array
    ref = lat.moments(f64=False)
    _same(first, ref)
    _same(second, ref)
    assert np.abs(ref["u"]).max() > 0
    lat.step(6)              # a new state, read again through the same array
    third = _noalloc(lat)
    _same(third, lat.moments(f64=False))
    assert not np.array_equal(third["u"], first["u"])
    _same(lat.moments_noalloc(), third)
    lat.close()


def test_noalloc_moments_reject_lattices_beyond_the_staging_array():
    side = int(round(lbm.NOALLOC_MAX_CELLS ** (1 / 3))) + 2
    assert side ** 3 > lbm.NOALLOC_MAX_CELLS
    lat = lbm.Lattice("D3Q19", (side, side, side), tau=0.6, storage="fp16")
    lat.init_equilibrium()
    out = np.empty(3 * lat.n, np.float32)
    rc = lbm.lib().lbm_vanse_moments_noalloc(lat.handle, None, None, out.ctypes.data)
    assert rc == -1
    msg = lbm.last_error()
    assert "at most" in msg and str(lbm.NOALLOC_MAX_CELLS) in msg
    # the handle keeps working, and a lattice at the limit is accepted
    assert lat.moments(f64=False)["rho"].shape == (lat.n,)
    lat.close()
    edge = lbm.Lattice("D2Q9", (lbm.NOALLOC_MAX_CELLS // 1024, 1024, 1), tau=0.6, storage="fp32")
    edge.init_equilibrium()
    assert edge.n <= lbm.NOALLOC_MAX_CELLS
    _same(_noalloc(edge), edge.moments(f64=False))
    edge.close()
