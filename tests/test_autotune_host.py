"""Host logic of the autotuner: size classes, keys and the JSON cache (no GPU)."""
import json

from paper_2108_13656_gb300 import autotune


def test_size_classes():
    assert autotune.size_class(1, 3840 * 2160) == "n1/p4^11"
    assert autotune.size_class(16, 100) == "n16/p4^3"
    assert autotune.size_class(17, 4 ** 7) == "n256/p4^7"
    assert autotune.size_class(300, 1) == "nmany/p4^0"


def test_key_separates_op_dtype_and_device():
    a = autotune.tuning_key("global", 0, 256, 8e8, "GB300")
    assert a != autotune.tuning_key("local", 0, 256, 8e8, "GB300")
    assert a != autotune.tuning_key("global", 2, 256, 8e8, "GB300")
    assert a != autotune.tuning_key("global", 0, 256, 8e8, "B200")


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    c = autotune.TuneCache(p)
    assert c.get("k") is None
    c.put("k", (8192, 2), {"8192,2": 12.5, "0,0": 14.0})
    assert autotune.TuneCache(p).get("k") == (8192, 2)
    with open(p) as f:
        d = json.load(f)
    assert d["k"]["us"]["0,0"] == 14.0


def test_cache_ignores_a_corrupt_file(tmp_path):
    p = tmp_path / "tune.json"
    p.write_text("{not json")
    assert autotune.TuneCache(str(p)).get("x") is None


def test_candidates_are_valid_tuning_values():
    for tc, cps in autotune.GLOBAL_CANDIDATES + autotune.LOCAL_CANDIDATES:
        assert tc == 0 or tc % 16 == 0
        assert 0 <= cps <= 8
    assert (0, 0) in autotune.LOCAL_CANDIDATES  # the library's own balanced width competes
