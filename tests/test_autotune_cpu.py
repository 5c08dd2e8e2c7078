"""The autotuner's choice and cache (host logic; the CUDA-event timing of the
batches is replaced by a fake timer): it takes the fastest of the 15
(tile, digit width) candidates, caches it per (device, size buckets, cameras,
mode), answers from the cache until forced, and survives a corrupt cache."""
import json
from types import SimpleNamespace

import torch

from paper_2412_00578_gb300 import autotune


def fake_batch(n=1_500_000, sizes=((640, 480), (1920, 1080))):
    scene = SimpleNamespace(means=torch.zeros(3, n))
    cams = [SimpleNamespace(width=w, height=h) for w, h in sizes]
    return scene, cams


def test_picks_the_fastest_candidate_and_caches_it(tmp_path):
    scene, cams = fake_batch()
    ms = {(t, d): 10.0 + t / 8 + (d or 8) / 10 for t, d in autotune.CANDIDATES}
    ms[(16, 6)] = 3.0
    calls = []

    def timer(tile, d):
        calls.append((tile, d))
        return ms[(tile, d)]

    path = tmp_path / "tune.json"
    a = autotune.tune(scene, cams, "cpu", cache_path=path, timer=timer, device_name="GB300 test")
    assert (a["tile"], a["sort_digit_bits"], a["ms"], a["cached"]) == (16, 6, 3.0, False)
    assert sorted(calls) == sorted(autotune.CANDIDATES) and len(a["timings"]) == 15
    # 8-bit digits are reported as 8 in the table and stored as 0 (automatic)
    assert "16/8" in a["timings"] and "16/0" not in a["timings"]
    b = autotune.tune(scene, cams, "cpu", cache_path=path, timer=timer, device_name="GB300 test")
    assert b["cached"] and (b["tile"], b["sort_digit_bits"]) == (16, 6) and len(calls) == 15
    cache = json.loads(path.read_text())
    assert list(cache) == [autotune.bucket_key("GB300 test", scene.means.shape[1], cams, "accutile")]
    # forced: timed again
    ms[(8, 0)] = 1.0
    c = autotune.tune(scene, cams, "cpu", cache_path=path, timer=timer, device_name="GB300 test", force=True)
    assert (c["tile"], c["sort_digit_bits"], c["cached"]) == (8, 0, False) and len(calls) == 30


def test_buckets_and_corrupt_cache(tmp_path):
    scene, cams = fake_batch()
    k = autotune.bucket_key("GB300 test", 1_500_000, cams, "accutile")
    assert k.startswith("GB300_test|n2^21|") and k.endswith("|v2|accutile")
    assert autotune.bucket_key("GB300 test", 1_500_000, cams, "snugbox") != k
    assert autotune.bucket_key("GB300 test", 3_000_000, cams, "accutile") != k
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    r = autotune.tune(scene, cams, "cpu", cache_path=path, timer=lambda t, d: float(t + (d or 8)),
                      device_name="GB300 test")
    assert (r["tile"], r["sort_digit_bits"], r["cached"]) == (8, 4, False)
    assert json.loads(path.read_text())[k]["tile"] == 8
