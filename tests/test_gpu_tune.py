"""The autotuner times candidate launch configurations and caches the best."""
import json

import pytest

from paper_2208_09267_gb300 import lbm, tune

pytestmark = pytest.mark.gpu


def test_step_tuner_picks_a_candidate_and_caches_it(tmp_path):
    cache = tune.Cache(str(tmp_path / "tune.json"))
    best, ms = tune.tune_step("D3Q19", "fp32", (64, 32, 32), steps=6, warmup=2, cache=cache,
                              blocks=[(32, 4), (64, 2)])
    assert set(ms) == {"row", "cell32x4", "cell64x2"}
    assert all(v > 0 for v in ms.values())
    assert best in ({"kernel": 2, "block": [0, 0]}, {"kernel": 1, "block": [32, 4]},
                    {"kernel": 1, "block": [64, 2]})
    data = json.load(open(tmp_path / "tune.json"))
    assert any(k.startswith("step/D3Q19/fp32") for k in data)
    # the cached choice is what a new lookup returns, without timing again
    kern, block = tune.best_config("D3Q19", "fp32", (64, 32, 32), tune.Cache(str(tmp_path / "tune.json")))
    assert kern == best["kernel"] and list(block) == best["block"]
    lat = lbm.Lattice("D3Q19", (64, 32, 32), kernel=kern, block=block)
    assert lat.row_kernel == (kern == 2)


def test_tile_tuner_times_batched_replays(tmp_path):
    from paper_2208_09267_gb300 import inputs
    cache = tune.Cache(str(tmp_path / "tune.json"))
    specs = inputs.batch_specs(count=6, d2_sides=(32, 64), d3_sides=(16, 24))
    best, ms = tune.tune_tiles(specs, steps=4, candidates=[1024, 4096], cache=cache)
    assert best in (1024, 4096) and set(ms) == {"1024", "4096"}
