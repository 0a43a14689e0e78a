"""The autotune cache file (host-only, no GPU): JSON entries keyed by device,
layout fingerprint and k; store is read-modify-write; a missing or corrupt
file reads as empty and is replaced on the next store."""
import json

import pytest

import paper_1708_07271_gb300 as bvg

CFG = {"pull_tile": 256, "pull_prefix": 1, "prefix_min_len": 8, "gather_pdl": 0, "col_block": 16, "pull_item": 4,
       "push_points": 1, "push_fused": 0, "pull_fused": 0}


def test_store_lookup_overwrite(tmp_path):
    path = tmp_path / "tune.json"
    assert bvg.bvg_autotune_cache_lookup(path, "dev/sm152/00ff/k1") is None  # no file yet
    bvg.bvg_autotune_cache_store(path, "dev/sm152/00ff/k1", CFG, 40.5, 100.25)
    other = dict(CFG, pull_tile=1024, col_block=32)
    bvg.bvg_autotune_cache_store(path, "dev/sm152/00ff/k8", other, 90.0, 200.0)
    assert bvg.bvg_autotune_cache_lookup(path, "dev/sm152/00ff/k1") == CFG
    assert bvg.bvg_autotune_cache_lookup(path, "dev/sm152/00ff/k8") == other
    assert bvg.bvg_autotune_cache_lookup(path, "dev/sm152/00ff/k2") is None
    doc = json.loads(path.read_text())  # the file is plain JSON
    assert doc["version"] == 1 and [e["key"] for e in doc["entries"]] == ["dev/sm152/00ff/k1", "dev/sm152/00ff/k8"]
    assert doc["entries"][0]["push_us"] == 40.5 and doc["entries"][0]["pull_us"] == 100.25
    new = dict(CFG, gather_pdl=1, push_points=0)
    bvg.bvg_autotune_cache_store(path, "dev/sm152/00ff/k1", new)
    assert bvg.bvg_autotune_cache_lookup(path, "dev/sm152/00ff/k1") == new
    assert bvg.bvg_autotune_cache_lookup(path, "dev/sm152/00ff/k8") == other


@pytest.mark.parametrize("text", ["", "{", "not json", '{"version": 1}', '{"entries": [{"key": "a"}]}',
                                  '{"entries": [{"key": "dev/x/k1", "pull_tile": 512}]}'])
def test_corrupt_file_reads_empty_and_is_replaced(tmp_path, text):
    path = tmp_path / "tune.json"
    path.write_text(text)
    assert bvg.bvg_autotune_cache_lookup(path, "dev/x/k1") is None
    bvg.bvg_autotune_cache_store(path, "dev/x/k1", CFG)
    assert bvg.bvg_autotune_cache_lookup(path, "dev/x/k1") == CFG
    assert len(json.loads(path.read_text())["entries"]) == 1


def test_file_written_by_hand_is_read(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"version": 1, "note": "hand-written", "entries": [
        {"key": "gpu/sm1/abc/k4", "pull_tile": 128, "pull_prefix": 0, "prefix_min_len": 16, "gather_pdl": 1,
         "col_block": 4, "pull_item": 16, "push_us": 1e2, "pull_us": 2.5e2}]}, indent=2))
    got = bvg.bvg_autotune_cache_lookup(path, "gpu/sm1/abc/k4")
    # a file without push_points, push_fused or pull_fused (written before those settings existed) reads them
    # as -1, the defaults
    assert got == {"pull_tile": 128, "pull_prefix": 0, "prefix_min_len": 16, "gather_pdl": 1, "col_block": 4,
                   "pull_item": 16, "push_points": -1, "push_fused": -1, "pull_fused": -1}


def test_bad_arguments(tmp_path):
    with pytest.raises(bvg.BvgError):
        bvg.bvg_autotune_cache_store(tmp_path / "t.json", "", CFG)
    with pytest.raises(bvg.BvgError):
        bvg.bvg_autotune_cache_store(tmp_path / "missing_dir" / "t.json", "k", CFG)
