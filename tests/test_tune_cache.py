"""The autotuner's cache, on the CPU (no GPU call): key layout and buckets,
store / save / load round trips, the fallback to the built-in heuristics when
no entry applies, and malformed or missing cache files."""
import json
import math

import pytest

import paper_1905_13038_gb300 as bz

GPU = "NVIDIA GB300/152"


@pytest.fixture(autouse=True)
def fresh_cache(tmp_path):
    bz.build()
    path = tmp_path / "tune.json"
    assert bz.tune_load(str(path)) == -1  # missing file: empty cache, saves go there
    yield path
    bz.tune_clear()


def test_key_layout_and_buckets():
    assert bz.tune_key(GPU, "window", 0, 15, 15, 3072, 4096) == f"{GPU}|window|0|h16|w16|s47"
    # next power of two of h and w; floor(2 log2(H W)) for the size
    for h, b in [(1, 1), (2, 2), (3, 4), (16, 16), (17, 32), (255, 256), (511, 512)]:
        assert bz.tune_key(GPU, "quantile", 1, h, 7, 10, 10).split("|")[3] == f"h{b}"
    for H, W in [(1, 1), (384, 512), (2048, 2048), (3508, 2480), (3072, 4096)]:
        s = int(bz.tune_key(GPU, "window", 1, 31, 31, H, W).split("|")[5][1:])
        assert s == math.floor(2 * math.log2(H * W))
    # neighbouring shapes share an entry, different precisions do not
    assert bz.tune_key(GPU, "window", 0, 63, 63, 3072, 4096) == bz.tune_key(GPU, "window", 0, 60, 50, 3000, 4200)
    assert bz.tune_key(GPU, "window", 0, 63, 63, 3072, 4096) != bz.tune_key(GPU, "window", 1, 63, 63, 3072, 4096)


def test_set_get_save_load_round_trip(fresh_cache):
    k1 = bz.tune_key(GPU, "window", 0, 15, 15, 3072, 4096)
    k2 = bz.tune_key(GPU, "quantile", 1, 101, 101, 2048, 2048)
    assert bz.tune_get(k1) is None
    bz.tune_set(k1, 26, 0.65, 0, 40.5)
    bz.tune_set(k2, 150, 1.0, -1, 180.25)
    assert bz.tune_get(k1) == {"tile_h": 26, "edge": pytest.approx(0.65), "stripes": 0, "us": pytest.approx(40.5)}
    assert bz.tune_save(None) == 0
    doc = json.loads(fresh_cache.read_text())  # plain JSON
    assert doc["version"] == 1 and set(doc["entries"]) == {k1, k2}
    bz.tune_clear()
    assert bz.tune_get(k1) is None
    assert bz.tune_load(str(fresh_cache)) == 2
    assert bz.tune_get(k2)["tile_h"] == 150


def test_bad_entries_are_refused():
    k = bz.tune_key(GPU, "window", 0, 15, 15, 3072, 4096)
    for args in [(-1, 0.5, 0), (10, 1.5, 0), (10, -0.1, 0), (10, 0.5, -2), (10, 0.5, 65)]:
        with pytest.raises(ValueError):
            bz.tune_set(k, *args)
    assert bz.tune_get(k) is None


def test_plan_falls_back_to_the_heuristic_without_an_entry():
    cached, plan = bz.tune_window_plan(GPU, "fp64", 3072, 4096, 15, 15, 152)
    assert not cached
    import ctypes
    L = bz._load()
    L.bz_tile_schedule.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
    L.bz_tile_schedule.restype = ctypes.c_int32
    out = (ctypes.c_int64 * 6)()
    # the heuristic schedule (pipelined kernel, no stripes) of the planner's own export
    assert L.bz_tile_schedule(3072, 4096, 152, 1, 0, out) == 0
    assert plan["tile_h"] == out[1] and plan["edge_h"] == out[2] and plan["n_edge"] == out[3]
    assert plan["tiles"] == out[4] <= plan["resident"] == 152 * 16
    # a tall window spanning five tile heights or more takes the stripe pre-pass
    assert bz.tune_window_plan(GPU, "fp64", 3072, 4096, 255, 255, 152)[1]["stripes"] == 1
    assert bz.tune_window_plan(GPU, "fp64", 3072, 4096, 63, 63, 152)[1]["stripes"] == 0
    assert bz.tune_window_plan(GPU, "fp64", 3072, 4096, 31, 127, 152)[1]["stripes"] == 0


def test_plan_follows_a_cached_entry():
    k = bz.tune_key(GPU, "window", 0, 63, 63, 3072, 4096)
    bz.tune_set(k, 32, 1.0, 0, 50.0)
    cached, plan = bz.tune_window_plan(GPU, "fp64", 3072, 4096, 63, 63, 152)
    assert cached and plan["tile_h"] == 32 and plan["n_edge"] == 0  # edge 1.0: uniform tiles
    assert plan["tiles"] == 16 * math.ceil(3072 / 32)
    bz.tune_set(k, 21, 1.0, 1, 50.0)  # stripes forced on (a 63-row window may take them)
    assert bz.tune_window_plan(GPU, "fp64", 3072, 4096, 63, 63, 152)[1]["stripes"] == 1
    # another precision or GPU does not see the entry
    assert not bz.tune_window_plan(GPU, "fp32", 3072, 4096, 63, 63, 152)[0]
    assert not bz.tune_window_plan("other/152", "fp64", 3072, 4096, 63, 63, 152)[0]
    # stripes are never taken for windows under 48 rows, whatever the entry says
    k15 = bz.tune_key(GPU, "window", 0, 15, 15, 3072, 4096)
    bz.tune_set(k15, 21, 1.0, 1, 40.0)
    assert bz.tune_window_plan(GPU, "fp64", 3072, 4096, 15, 15, 152)[1]["stripes"] == 0


@pytest.mark.parametrize("text", [
    "", "{", "not json", "[]", '{"version": 2, "entries": {}}',
    '{"version": 1, "entries": {"k": {"tile_h": 21, "edge": 0.8, "stripes": 0}}}',          # field missing
    '{"version": 1, "entries": {"k": {"tile_h": 21, "edge": 0.8, "stripes": 0, "us": 1, "x": 2}}}',
    '{"version": 1, "entries": {"k": {"tile_h": 21, "edge": 7, "stripes": 0, "us": 1}}}',   # out of range
    '{"version": 1, "entries": {"k": {"tile_h": 21, "edge": 0.8, "stripes": 0, "us": 1}}} trailing',
    '{"version": 1}',
])
def test_malformed_cache_file_reads_as_empty(fresh_cache, text):
    k = bz.tune_key(GPU, "window", 0, 15, 15, 3072, 4096)
    fresh_cache.write_text(text.replace('"k"', json.dumps(k)))
    assert bz.tune_load(str(fresh_cache)) == -2
    assert bz.tune_get(k) is None
    assert not bz.tune_window_plan(GPU, "fp64", 3072, 4096, 15, 15, 152)[0]
    # the next save rewrites the file whole and valid
    bz.tune_set(k, 22, 0.82, 0, 41.0)
    assert bz.tune_save(None) == 0
    assert bz.tune_load(str(fresh_cache)) == 1
