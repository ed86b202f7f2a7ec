"""The autotuner times candidate launch configurations, caches the best, and
the solver's handles launch what the cache holds."""
import json

import numpy as np
import pytest

from paper_2208_09267_gb300 import lbm, tune

pytestmark = pytest.mark.gpu


def test_step_tuner_picks_a_candidate_and_caches_it(tmp_path):
    cache = tune.Cache(str(tmp_path / "tune.json"), seed=None)
    best, ms = tune.tune_step("D3Q19", "fp32", (256, 32, 32), steps=6, warmup=2, cache=cache,
                              blocks=[(32, 4), (64, 2)], row_shapes=[(0, 0), (5, 2), (6, 3)])
    assert {"row7x3", "row5x2", "row6x3", "cell32x4", "cell64x2"} <= set(ms)
    assert all(v > 0 for v in ms.values())
    name = min(ms, key=ms.get)
    assert best["kernel"] == (2 if name.startswith("row") else 1)
    data = json.load(open(tmp_path / "tune.json"))
    assert any(k.startswith("step/D3Q19/fp32") for k in data)
    hit = tune.best_config("D3Q19", "fp32", (256, 32, 32), cache=tune.Cache(str(tmp_path / "tune.json"),
                                                                                seed=None))
    assert hit["kernel"] == best["kernel"] and hit["row_shape"] == best["row_shape"]


@pytest.mark.parametrize("entry,expect", [
    ({"kernel": 2, "block": [0, 0], "row_shape": [5, 2]}, {"kernel": "row", "consumers": 5, "stages": 2}),
    ({"kernel": 2, "block": [0, 0], "row_shape": [6, 3]}, {"kernel": "row", "consumers": 6, "stages": 3}),
    ({"kernel": 1, "block": [64, 2], "row_shape": None}, {"kernel": "cell", "block": [64, 2]})])
def test_cached_choice_changes_the_launched_variant(tmp_path, monkeypatch, entry, expect):
    """A handle created with tuned=True launches the cached shape of its size
    bucket, and steps to the same state as the default shape (the shape does
    not change the arithmetic of the row kernel; the cell kernel rounds in
    its own order)."""
    path = tmp_path / "tune.json"
    shape = (256, 24, 20)
    key = "step/" + tune.bucket_key("D3Q19", "fp32", shape)
    path.write_text(json.dumps({key: {"best": entry, "ms": {}}}))
    monkeypatch.setenv("LBM_TUNE_CACHE", str(path))
    monkeypatch.setattr(tune, "SEED_CACHE", None)
    tuned = lbm.Lattice("D3Q19", shape, tau=0.6, storage="fp32")
    plain = lbm.Lattice("D3Q19", shape, tau=0.6, storage="fp32", tuned=False)
    assert tuned.tuned_from == key and plain.tuned_from is None
    got = tuned.launch_shape
    assert {k: got[k] for k in expect} == expect
    assert plain.launch_shape["kernel"] == "row" and plain.launch_shape["consumers"] == 7
    eps = 0.6 + 0.3 * np.random.default_rng(3).random(int(np.prod(shape)))
    for lat in (tuned, plain):
        lat.set_epsilon(eps.astype(np.float32))
        lat.set_force((1e-5, 0, 0))
        lat.init_equilibrium()
        lat.step(21)
    pt, pp = tuned.populations(), plain.populations()
    if expect["kernel"] == "row":
        assert np.array_equal(pt, pp)
    else:
        assert np.abs(pt - pp).max() <= 1e-6 * np.abs(pp).max()


def test_tile_tuner_times_batched_replays(tmp_path):
    from paper_2208_09267_gb300 import inputs
    cache = tune.Cache(str(tmp_path / "tune.json"), seed=None)
    specs = inputs.batch_specs(count=6, d2_sides=(32, 64), d3_sides=(16, 24))
    best, ms = tune.tune_tiles(specs, steps=4, candidates=[1024, 4096], cache=cache)
    assert best in (1024, 4096) and set(ms) == {"1024", "4096"}
