"""The autotune cache of batch plans (host code of the library, no GPU): the JSON file it
writes, lookups, replacement, refusals, and that a file it cannot parse is left alone."""
import json

import pytest

import paper_1811_11785_gb300 as sp


@pytest.fixture()
def cache(tmp_path):
    path = tmp_path / "tune.json"
    sp.set_tune_cache(path)
    yield path
    sp.set_tune_cache(None)


def test_missing_file_is_an_empty_cache(cache):
    assert not cache.exists()
    assert sp.tune_cache_get("sm103-152sm/mode1/prec1/n4/0123456789abcdef") is None


def test_round_trip_and_file_format(cache):
    sp.tune_cache_put("b/key", 8, 2, 1, 1.25, grouped=1)
    sp.tune_cache_put("a/key", 32, 1, 0, 8.5)
    assert sp.tune_cache_get("a/key") == dict(branches=32, tiles_per_cta=1, proj_variant=0, ms=8.5, grouped=0)
    assert sp.tune_cache_get("b/key") == dict(branches=8, tiles_per_cta=2, proj_variant=1, ms=1.25, grouped=1)
    doc = json.loads(cache.read_text())
    assert doc["format"] == "svdphat-tune-cache" and doc["version"] == 1
    assert list(doc["plans"]) == ["a/key", "b/key"]          # sorted by key
    assert doc["plans"]["b/key"] == {"branches": 8, "tiles_per_cta": 2, "proj_variant": 1, "grouped": 1, "ms": 1.25}
    assert [p.name for p in cache.parent.iterdir()] == ["tune.json"]   # no temporary file left


def test_replace_keeps_other_entries(cache):
    sp.tune_cache_put("k1", 8, 1, 0, 2.0)
    sp.tune_cache_put("k2", 32, 4, 0, 3.0)
    sp.tune_cache_put("k1", 128, 2, 1, 1.5)
    assert sp.tune_cache_get("k1") == dict(branches=128, tiles_per_cta=2, proj_variant=1, ms=1.5, grouped=0)
    assert sp.tune_cache_get("k2") == dict(branches=32, tiles_per_cta=4, proj_variant=0, ms=3.0, grouped=0)


def test_reads_a_file_written_by_another_program(cache):
    cache.write_text(json.dumps({"format": "svdphat-tune-cache", "version": 1,
                                 "plans": {"x": {"ms": 4.0, "proj_variant": 0, "tiles_per_cta": 4,
                                                 "branches": 16}}}, indent=4))
    assert sp.tune_cache_get("x") == dict(branches=16, tiles_per_cta=4, proj_variant=0, ms=4.0, grouped=0)   # absent: 0
    sp.tune_cache_put("y", 8, 1, 0, 1.0)
    assert set(json.loads(cache.read_text())["plans"]) == {"x", "y"}


@pytest.mark.parametrize("key", ["", 'a"b', "a\\b", "tab\there", "x" * 513])
def test_bad_keys_are_refused(cache, key):
    with pytest.raises(sp.SvdPhatError):
        sp.tune_cache_put(key, 8, 1, 0, 1.0)
    assert not cache.exists()


@pytest.mark.parametrize("shape", [(0, 1, 0, 1.0), (8, 3, 0, 1.0), (8, 1, 2, 1.0), (8, 1, 0, -1.0), (8, 1, 0, 1.0, 2)])
def test_bad_shapes_are_refused(cache, shape):
    with pytest.raises(sp.SvdPhatError):
        sp.tune_cache_put("k", *shape)


@pytest.mark.parametrize("text", ["not json", '{"plans": {}}', '{"format": "svdphat-tune-cache", "plans": {"k": 3}}',
                                  '{"format": "svdphat-tune-cache", "plans": {"k": {"branches": 8}}}'])
def test_a_file_that_does_not_parse_is_left_alone(cache, text):
    cache.write_text(text)
    with pytest.raises(sp.SvdPhatError):
        sp.tune_cache_get("k")
    with pytest.raises(sp.SvdPhatError):
        sp.tune_cache_put("k", 8, 1, 0, 1.0)
    assert cache.read_text() == text


def test_disabled_cache_stores_nothing(tmp_path):
    sp.set_tune_cache(None)
    sp.tune_cache_put("k", 8, 1, 0, 1.0)
    assert sp.tune_cache_get("k") is None
    assert list(tmp_path.iterdir()) == []
