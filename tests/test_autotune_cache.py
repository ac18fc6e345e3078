"""Host side of the autotuner: its cache keys and the JSON cache (no GPU needed).  The search
itself runs in tests/test_gpu_autotune.py."""
from paper_1712_09407_gb300 import autotune


def test_cache_keys_by_device_and_size_class():
    assert autotune.cache_key("NVIDIA GB300", 3_300_000) == "NVIDIA GB300|2^21"
    assert autotune.cache_key("NVIDIA GB300", 1) == "NVIDIA GB300|2^0"
    assert autotune.cache_key("NVIDIA GB300", 2 ** 21) != autotune.cache_key("NVIDIA GB300", 2 ** 21 - 1)


def test_cache_round_trip_keeps_other_keys(tmp_path):
    path = str(tmp_path / "t.json")
    assert autotune.load(path, "a") is None
    a = {"bin_occupancy": 0.5, "neighbours_block": 256, "construct_block": 128}
    b = {"bin_occupancy": 2.0, "neighbours_block": 128, "construct_block": 64}
    autotune.store(path, "a", a)
    autotune.store(path, "b", b)
    assert autotune.load(path, "a") == a and autotune.load(path, "b") == b


def test_search_space_fields_are_tuning_fields():
    from paper_1712_09407_gb300.tracker import tpc_tuning
    names = {f for f, _ in tpc_tuning._fields_}
    for field, values, stages in autotune.SPACE:
        assert field in names and values and set(stages) <= set(autotune.STAGES)
