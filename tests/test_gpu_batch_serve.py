"""Batched stepping and the continuous-batching server on the GPU."""
import numpy as np
import pytest

from paper_2208_09267_gb300 import inputs as I
from paper_2208_09267_gb300 import lbm, serve

pytestmark = pytest.mark.gpu


def _lattice(spec, storage, kernel="cell"):
    nz, ny, nx = spec.shape
    lat = lbm.Lattice(spec.lattice, (nx, ny, nz), tau=spec.tau, storage=storage, kernel=kernel)
    lat.set_epsilon(spec.eps().ravel().astype(np.float32))
    lat.set_force(spec.g)
    lat.init_equilibrium()
    return lat


def _specs():
    return [I.LatticeSpec("D2Q9", (1, 40, 52), 0.61, 0.2, 7),
            I.LatticeSpec("D3Q19", (12, 10, 14), 0.9, 0.1, 8),
            I.LatticeSpec("D2Q9", (1, 33, 31), 1.1, 0.3, 9),
            I.LatticeSpec("D3Q19", (9, 16, 20), 0.56, 0.05, 10),
            I.LatticeSpec("D3Q27", (8, 9, 10), 0.7, 0.15, 11)]


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_batch_equals_each_lattice_alone(storage):
    """Members of one batch (different lattices, sizes, tau) advance exactly
    as each would alone: the per-cell arithmetic does not see the batch."""
    specs = _specs()
    budgets = [40, 40, 26, 40, 12]
    batched = [_lattice(s, storage) for s in specs]
    alone = [_lattice(s, storage) for s in specs]
    b = lbm.Batch(max_members=8, max_tiles=64, tile_cells=512)
    for lat, k in zip(batched, budgets):
        b.add(lat, k)
    b.step(10)
    b.step(10, check=True)
    b.step(20, check=True)
    for lat, k in zip(alone, budgets):
        lat.step(k)
    for s, lb, la, k in zip(specs, batched, alone, budgets):
        assert lb.steps_done == k
        assert np.array_equal(lb.populations(), la.populations()), s
    st = b.stats(batched[0])
    assert st["steps_done"] == 40 and st["mass"] > 0
    assert st["residual"] >= 0  # two checks seen


def _row_specs():
    # row pitch classes 64, 128, 256 and 512, ragged rows, walls on y and z
    return [I.LatticeSpec("D2Q9", (1, 40, 52), 0.61, 0.2, 7),
            I.LatticeSpec("D3Q19", (12, 10, 14), 0.9, 0.1, 8),
            I.LatticeSpec("D2Q9", (1, 33, 100), 1.1, 0.3, 9),
            I.LatticeSpec("D3Q19", (9, 16, 200), 0.56, 0.05, 10),
            I.LatticeSpec("D3Q27", (8, 9, 10), 0.7, 0.15, 11),
            I.LatticeSpec("D2Q9", (1, 12, 300), 0.8, 0.1, 12)]


def _row_lattice(spec, storage, kernel, walls=0):
    nz, ny, nx = spec.shape
    lat = lbm.Lattice(spec.lattice, (nx, ny, nz), tau=spec.tau, storage=storage, kernel=kernel,
                      walls=walls)
    lat.set_epsilon(spec.eps().ravel().astype(np.float32))
    lat.set_force(spec.g)
    lat.init_equilibrium()
    return lat


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_batched_row_kernel_equals_each_lattice_alone(storage):
    """Members created for the row-staged kernel are stepped by the batched
    row kernel: bit-identical to each lattice stepped alone by the row
    kernel (members of every row-pitch class, walls, different budgets and
    parities), and the check sums agree with the lattice's own."""
    specs = _row_specs()
    walls = [0, 2, 0, 4, 6, 2]
    budgets = [40, 40, 26, 40, 13, 33]
    batched = [_row_lattice(s, storage, "row", w) for s, w in zip(specs, walls)]
    alone = [_row_lattice(s, storage, "row", w) for s, w in zip(specs, walls)]
    cell = [_row_lattice(s, storage, "cell", w) for s, w in zip(specs, walls)]
    for group in (batched, alone, cell):
        group[4].step(3)      # an odd start: this member runs at the other parity
    b = lbm.Batch(max_members=8, max_tiles=64, tile_cells=512)
    for lat, k in zip(batched, budgets):
        b.add(lat, k)
    b.step(10)
    b.step(10, check=True)
    b.step(20, check=True)
    for lat, k in zip(alone, budgets):
        lat.step(k)
    for lat, k in zip(cell, budgets):
        lat.step(k)
    differs = 0
    for s, lb, la, lc in zip(specs, batched, alone, cell):
        assert lb.steps_done == la.steps_done
        pb = lb.populations()
        assert np.array_equal(pb, la.populations()), s
        differs += not np.array_equal(pb, lc.populations())
    assert differs >= 1   # the cell kernel rounds differently: the row path ran
    st = b.stats(batched[0])
    assert st["steps_done"] == 40 and st["step_of_stats"] == 39
    # the same sums, added in another order
    ref = _row_lattice(specs[0], storage, "row", walls[0])
    ref.step(39)
    st2 = ref.step(1)
    assert abs(st["mass"] - st2["mass"]) <= 1e-12 * abs(st2["mass"])
    assert st["residual"] >= 0


@pytest.mark.parametrize("kernel", ["row", "cell"])
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_batch_member_with_phi_refresh_equals_alone(kernel, storage):
    """A member whose phi is refreshed between replays (set_epsilon with a
    time derivative) advances exactly as the same lattice alone: the step
    after the refresh decodes with the old shift, every later step of the
    replay with the new one."""
    specs = _row_specs()[:2]
    g = np.random.default_rng(5)
    lats, refs = [], []
    for s in specs:
        nz, ny, nx = s.shape
        for group in (lats, refs):
            group.append(_row_lattice(s, storage, kernel))
    b = lbm.Batch(max_members=4, max_tiles=64)
    for lat in lats:
        b.add(lat, 60)
    b.step(10)
    for ref in refs:
        ref.step(10)
    for lat, ref in zip(lats, refs):
        n = lat.n
        e = (0.6 + 0.3 * g.random(n)).astype(np.float32)
        de = (1e-4 * g.standard_normal(n)).astype(np.float32)
        lat.set_epsilon(e, de, 10)
        ref.set_epsilon(e, de, 10)
    b.step(20)
    for ref in refs:
        ref.step(20)
    for lat, ref in zip(lats, refs):
        assert lat.steps_done == ref.steps_done == 30
        assert np.array_equal(lat.populations(), ref.populations())


def test_batch_members_join_and_leave():
    specs = _specs()[:3]
    lats = [_lattice(s, "fp16") for s in specs]
    ref = [_lattice(s, "fp16") for s in specs]
    b = lbm.Batch(max_members=4, max_tiles=64)
    b.add(lats[0], 100)
    b.step(20)
    b.add(lats[1], 100)          # joins while member 0 is running
    b.step(20)
    b.remove(lats[0])
    b.add(lats[2], 30)
    b.step(40)
    ref[0].step(40)
    ref[1].step(60)
    ref[2].step(30)
    for a, r in zip(lats, ref):
        assert a.steps_done == r.steps_done
        assert np.array_equal(a.populations(), r.populations())


def _requests(count, rate=200.0):
    reqs = serve.make_requests(rate, count, seed_offset=7100, sides=(16, 40), steps=(60, 400),
                               residual_share=0.0)
    return reqs


def test_server_result_is_the_same_alone_and_in_the_mix():
    """Requests that arrive while others run join the batch; each result
    equals the result of serving that request alone."""
    reqs = _requests(6)
    srv = serve.Server(storage="fp16", hbm_budget=8e9, macro_steps=20)
    summary = srv.run(reqs)
    srv.close()
    assert summary["completed"] == 6 and summary["peak_members"] >= 2
    for r in reqs:
        solo = serve.Request(r.rid, r.spec, 0.0, r.eps)
        s1 = serve.Server(storage="fp16", hbm_budget=8e9, macro_steps=20)
        s1.run([solo])
        s1.close()
        assert solo.steps_done == r.steps_done
        for key in ("u", "p"):
            assert np.array_equal(solo.result[key], r.result[key]), (r.rid, key)


def test_server_admits_by_budget_and_retires_on_residual():
    reqs = _requests(5)
    sizes = sorted(serve.request_bytes(r.spec, "fp16") for r in reqs)
    budget = sizes[-1] + sizes[-2]
    srv = serve.Server(storage="fp16", hbm_budget=budget, macro_steps=20)
    summary = srv.run(reqs)
    srv.close()
    assert summary["completed"] == 5
    assert 0 < summary["peak_bytes"] <= budget and summary["peak_members"] < 5
    # a channel flow converges: the residual target retires it early
    spec = I.LatticeSpec("D2Q9", (1, 34, 32), 0.8, 0.0, 1, steps=200000, residual_tol=1e-6)
    req = serve.Request(0, spec, 0.0, np.ones(34 * 32))
    srv = serve.Server(storage="fp32", hbm_budget=1e9, macro_steps=200)
    srv.run([req])
    srv.close()
    assert req.status == "converged" and req.steps_done < 200000


def test_fp16_served_result_close_to_fp32_alone():
    """The FP16-shifted served answer (stochastic rounding) stays within 2e-3
    (relative L2) of the FP32 answer of the same request, on the served
    workload's step budgets."""
    reqs = serve.make_requests(200.0, 3, seed_offset=7300, sides=(24, 48), steps=(500, 1500),
                               residual_share=0.0)
    srv = serve.Server(storage="fp16", hbm_budget=8e9, macro_steps=20)
    srv.run(reqs)
    srv.close()
    for r in reqs:
        ref = serve.Request(r.rid, r.spec, 0.0, r.eps)
        serve.run_sequential([ref], storage="fp32", check_every=20)
        for key in ("u",):
            a, b = r.result[key].astype(np.float64), ref.result[key].astype(np.float64)
            assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 2e-3
