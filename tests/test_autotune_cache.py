"""Host logic of the autotuner's cache (no GPU): results survive a save and
load, a missing or corrupt cache file reads as empty instead of failing, and
a save replaces the file atomically (no partial file is left behind)."""
import json
import os

from paper_2109_14704_gb300 import autotune


def test_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "cache.json")
    cache = {"GB300|32768|8|1024": {"fwd": [12, 4, 0], "inv": [12, 3, 0]}}
    autotune._save_cache(path, cache)
    assert autotune._load_cache(path) == cache


def test_missing_and_corrupt_files_read_as_empty(tmp_path):
    assert autotune._load_cache(str(tmp_path / "absent.json")) == {}
    bad = tmp_path / "bad.json"
    bad.write_text("{ not json")
    assert autotune._load_cache(str(bad)) == {}


def test_save_leaves_no_temporary(tmp_path):
    path = str(tmp_path / "cache.json")
    autotune._save_cache(path, {"a": 1})
    autotune._save_cache(path, {"a": 2})
    assert sorted(os.listdir(tmp_path)) == ["cache.json"]
    assert json.loads(open(path).read()) == {"a": 2}
