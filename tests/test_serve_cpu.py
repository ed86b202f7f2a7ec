"""Host logic of the server (admission, retirement, rejection) against a
fake device layer: no GPU involved."""
import numpy as np

from paper_2208_09267_gb300 import inputs as I
from paper_2208_09267_gb300 import serve


class FakeLattice:
    def __init__(self, lattice, shape, tau=0.6, storage="fp16", stream=None, fp16_scale_log2=10):
        self.n = int(np.prod(shape))
        self.steps = 0
        self.closed = False

    def set_epsilon(self, e):
        pass

    def set_force(self, g):
        pass

    def init_equilibrium(self):
        pass

    def moments(self, f64=False):
        return {"u": np.zeros((3, self.n)), "p": np.zeros(self.n)}

    def moments_noalloc(self):
        self.read_without_allocation = True
        return self.moments()

    def close(self):
        self.closed = True


class FakeBatch:
    def __init__(self, **kw):
        self.members = {}

    def add(self, lat, budget):
        self.members[id(lat)] = [lat, budget]

    def remove(self, lat):
        del self.members[id(lat)]

    def step(self, k, check=False):
        for m in self.members.values():
            s = min(k, m[1])
            m[0].steps += s
            m[1] -= s

    def stats(self, lat):
        lt = self.members[id(lat)][0]
        # a residual that falls by 10x per macro-step
        return {"steps_done": lt.steps, "residual": 10.0 ** (-lt.steps / 10), "nan_seen": False}

    def close(self):
        pass


def _patch(monkeypatch):
    monkeypatch.setattr(serve.lbm, "Lattice", FakeLattice)
    monkeypatch.setattr(serve.lbm, "Batch", FakeBatch)
    monkeypatch.setattr(serve, "request_bytes", lambda spec, storage: spec.cells)


def _req(rid, side, steps, arrival=0.0, tol=0.0):
    spec = I.LatticeSpec("D3Q19", (side, side, side), 0.6, 0.1, rid, steps=steps, residual_tol=tol)
    return serve.Request(rid, spec, arrival, np.ones(spec.cells))


def test_fifo_admission_respects_the_budget(monkeypatch):
    _patch(monkeypatch)
    reqs = [_req(j, 10, 40) for j in range(5)]   # 1000 "bytes" each
    srv = serve.Server(hbm_budget=2500, macro_steps=20)
    summary = srv.run(reqs)
    assert summary["completed"] == 5
    assert summary["peak_members"] == 2
    assert all(r.status == "done" and r.steps_done == 40 for r in reqs)
    assert srv.used == 0


def test_oversized_request_is_rejected_not_blocking(monkeypatch):
    _patch(monkeypatch)
    reqs = [_req(0, 20, 40), _req(1, 10, 40)]      # 8000 > budget
    srv = serve.Server(hbm_budget=5000, macro_steps=20)
    summary = srv.run(reqs)
    assert reqs[0].status == "rejected" and reqs[1].status == "done"
    assert summary["rejected"] == 1 and summary["completed"] == 1


def test_residual_target_retires_early(monkeypatch):
    _patch(monkeypatch)
    r = _req(0, 8, 10000, tol=1e-5)
    srv = serve.Server(hbm_budget=10 ** 6, macro_steps=20)
    srv.run([r])
    assert r.status == "converged" and r.steps_done < 100


def test_macro_steps_must_be_even(monkeypatch):
    _patch(monkeypatch)
    import pytest
    with pytest.raises(ValueError):
        serve.Server(macro_steps=7)
