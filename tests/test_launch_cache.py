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


def test_shipped_cache_holds_complete_valid_shapes():
    """Every stored entry names each launch field once, within the ranges
    cg_set_launch accepts, under a well-formed key."""
    data = cg._read_launch_cache(cg.LAUNCH_CACHE)
    assert data, "the package ships tuned shapes"
    fields = {f for f, _ in cg.cg_launch._fields_}
    for key, shape in data.items():
        gpu, prec, rb, nb, l2 = key.split("|")
        assert gpu and prec in ("f32", "f64") and l2 in ("l2cold", "l2warm")
        assert rb.startswith("R~") and nb.startswith("N~")
        for b in (int(rb[2:]), int(nb[2:])):
            assert b >= 1 and b & (b - 1) == 0
        assert set(shape) == fields
        assert 1 <= shape["repair_blocks_per_sm"] <= 64 and 1 <= shape["check_blocks_per_sm"] <= 64
        for f in ("dir_blocks_per_sm", "geom_blocks_per_sm", "test_blocks_per_sm"):
            assert 0 <= shape[f] <= 64
        assert shape["dir_low_priority"] in (0, 1) and shape["dir_beside_geom"] in (0, 1)
        assert 0 <= shape["ring_order"] <= 7
