"""Host logic of the tile-shape autotuner (no GPU): cache keys and the JSON
cache round trip."""

import os

import erpp_inputs as I


def test_workload_key_classes():
    from paper_1405_6969_gb300 import autotune
    p = I.CFG_CUBE256.params()
    k1 = autotune.workload_key(p, 1_000_000)
    k2 = autotune.workload_key(p, 1_100_000)  # same density class
    k3 = autotune.workload_key(p, 4_000_000)  # two classes denser
    k4 = autotune.workload_key(p, 1_000_000, kahan=True)
    assert k1 == k2 and k1 != k3 and k1 != k4
    assert k1.startswith("256x256x256|cp=3.0,3.0,3.0|")


def test_cache_round_trip(tmp_path):
    from paper_1405_6969_gb300 import autotune
    path = os.path.join(tmp_path, "sub", "tune.json")
    assert autotune.load_cache(path) == {}
    autotune.save_cache(path, {"k": {"tile": [16, 4], "ms": {"16x4": 1.0}}})
    assert autotune.load_cache(path)["k"]["tile"] == [16, 4]
    with open(path, "w") as f:
        f.write("not json")
    assert autotune.load_cache(path) == {}
