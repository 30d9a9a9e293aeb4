"""Persisted launch shapes (host logic): the cache key buckets problems by
GPU model, precision, replica count and cell count, and the file keeps every
entry written to it."""
import json

import paper_1702_02939_gb300 as cg


def test_key_buckets_cell_and_replica_counts():
    k = cg.launch_cache_key("NVIDIA GB300", 262144, 1, 0, 256 << 20)
    assert k == "NVIDIA GB300|f64|R~1|N~262144|l2cold"
    assert cg.launch_cache_key("NVIDIA GB300", 250000, 1, 0, 1) == k  # nearest power of two
    assert cg.launch_cache_key("NVIDIA GB300", 262144, 1, 1, 0) == "NVIDIA GB300|f32|R~1|N~262144|l2warm"
    assert cg.launch_cache_key("NVIDIA GB300", 2012412, 512, 0, 0).startswith("NVIDIA GB300|f64|R~512|N~2097152")
    assert cg.launch_cache_key("A|B", 64, 1, 0, 0).startswith("A/B|")  # the separator stays unambiguous


def test_cache_file_round_trip(tmp_path):
    path = str(tmp_path / "cache.json")
    assert cg._read_launch_cache(path) == {}
    cg._write_launch_cache(path, "a", {"repair_blocks_per_sm": 4, "ring_order": 1})
    cg._write_launch_cache(path, "b", {"repair_blocks_per_sm": 8})
    data = cg._read_launch_cache(path)
    assert data == {"a": {"repair_blocks_per_sm": 4, "ring_order": 1}, "b": {"repair_blocks_per_sm": 8}}
    with open(path, "w") as f:
        f.write("not json")
    assert cg._read_launch_cache(path) == {}
    with open(path, "w") as f:
        json.dump([1, 2], f)
    assert cg._read_launch_cache(path) == {}
