"""Host logic of the autotuner (no GPU): size buckets, the JSON cache and the
lookups that fall back to the library defaults."""
import json

from paper_2208_09267_gb300 import tune


def test_bucket_key_groups_sizes_by_power_of_two_and_row_fill():
    k = tune.bucket_key
    assert k("D3Q19", "fp32", (128, 128, 128)) == "D3Q19/fp32/b21/x32"
    # same power of two of cells, same row-fill class: same bucket
    assert k("D3Q19", "fp32", (64, 128, 300)) == k("D3Q19", "fp32", (96, 200, 150))
    # nx not a multiple of 32 is its own class
    assert k("D3Q19", "fp32", (100, 128, 128)).endswith("/xr")
    # lattice and storage are part of the key; 2D shapes may omit nz
    assert k("D2Q9", "fp16", (64, 64)) == "D2Q9/fp16/b12/x32"
    assert k("D3Q19", "fp16", (128, 128, 128)) != k("D3Q19", "fp32", (128, 128, 128))


def test_cache_round_trip_and_defaults(tmp_path):
    path = str(tmp_path / "sub" / "autotune.json")
    c = tune.Cache(path, seed=None)
    shape = (256, 64, 64)
    # empty cache: the library's own choices
    assert tune.best_config("D3Q19", "fp32", shape, cache=c) is None
    assert tune.best_block("D3Q19", "fp32", shape, cache=c) == (0, 0)
    assert tune.best_tile("fp16", cache=c) is None
    key = tune.bucket_key("D3Q19", "fp32", shape)
    c.put("step/" + key, {"best": {"kernel": 2, "block": [0, 0], "row_shape": [5, 2]},
                          "ms": {"row5x2": 0.5}})
    c.put("block/" + key, {"best": [128, 1], "ms": {"128x1": 0.7}})
    c.put("tile/fp16/n256", {"best": 8192, "ms": {"8192": 1.0}})
    # persisted: a fresh instance reads what was written
    c2 = tune.Cache(path, seed=None)
    hit = tune.best_config("D3Q19", "fp32", shape, cache=c2)
    assert (hit["kernel"], hit["row_shape"], hit["key"]) == (2, [5, 2], "step/" + key)
    assert tune.best_block("D3Q19", "fp32", shape, cache=c2) == (128, 1)
    assert tune.best_tile("fp16", cache=c2) == {"best": 8192, "key": "tile/fp16/n256"}
    # another lattice of the same bucket reuses the entry; another bucket does not
    assert tune.best_block("D3Q19", "fp32", (128, 128, 64), cache=c2) == (128, 1)
    assert tune.best_block("D3Q19", "fp32", (256, 256, 256), cache=c2) == (0, 0)
    assert tune.best_config("D3Q19", "fp16", shape, cache=c2) is None
    with open(path) as fh:
        assert set(json.load(fh)) == {"step/" + key, "block/" + key, "tile/fp16/n256"}


def test_seed_file_is_read_first_and_overlaid(tmp_path):
    seed = tmp_path / "seed.json"
    seed.write_text(json.dumps({"tile/fp32/n8": {"best": 2048}, "tile/fp16/n8": {"best": 1024}}))
    local = tmp_path / "local.json"
    local.write_text(json.dumps({"tile/fp16/n8": {"best": 4096}}))
    c = tune.Cache(str(local), seed=str(seed))
    assert tune.best_tile("fp32", cache=c)["best"] == 2048
    assert tune.best_tile("fp16", cache=c)["best"] == 4096


def test_environment_selects_the_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("LBM_TUNE_CACHE", str(tmp_path / "env.json"))
    assert tune.Cache(seed=None).path == str(tmp_path / "env.json")


def test_unreadable_cache_starts_empty(tmp_path):
    path = tmp_path / "autotune.json"
    path.write_text("{not json")
    c = tune.Cache(str(path), seed=None)
    assert c.data == {}
    c.put("block/x", {"best": [32, 1], "ms": {}})
    assert json.loads(path.read_text()) == {"block/x": {"best": [32, 1], "ms": {}}}
