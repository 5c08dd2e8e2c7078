"""The sort's plan (gs_sort_plan_for, the host form of the plan every sort
kernel evaluates on the device): the key image (tile << w) | (depth bits -
least) keeps the keys' order with w the bit length of the depth span, the
digits cover the image's bits with the fewest passes the digit width allows,
a stand-alone gs_sort runs an even count, and gs_forward's emit starts from
the buffer that makes the last pass end in buffer 0."""
import numpy as np
import pytest

from paper_2412_00578_gb300 import build

build.build()
from paper_2412_00578_gb300 import raster  # noqa: E402


def tile_bits(tiles):
    return max(int(tiles) - 1, 0).bit_length()


def test_edge_cases():
    # no range recorded: all 32 depth bits
    assert raster.sort_plan_for(4240, 1, 0)[2] == 32
    # one depth for the whole frame: no depth bits, tile bits only
    p, d, w, s = raster.sort_plan_for(4240, 0x3F800000, 0x3F800000)
    assert w == 0 and p * d >= 13 and p == 2 and s == 0
    # one tile and one depth: nothing to sort, still two (identity) passes
    p, d, w, s = raster.sort_plan_for(1, 7, 7)
    assert (p, d, w, s) == (2, 0, 0, 0)
    # the 3M frame's range: 13 tile bits + 26 depth bits
    assert raster.sort_plan_for(80 * 53, 0x3F69DDE0, 0x42D1EB09) == (5, 8, 26, 1)
    assert raster.sort_plan_for(80 * 53, 0x3F69DDE0, 0x42D1EB09, fused=False) == (6, 7, 26, 0)
    with pytest.raises(raster.GsError):
        raster.sort_plan_for(0, 0, 1)
    with pytest.raises(raster.GsError):
        raster.sort_plan_for(16, 0, 1, sort_digit_bits=9)


def test_plan_rules_on_random_frames():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        tiles = int(rng.integers(1, 1 << 20))
        least = int(rng.integers(1, 0x7F000000))
        greatest = least + int(rng.integers(0, 1 << int(rng.integers(0, 31))))
        greatest = min(greatest, 0x7F7FFFFF)
        digits = int(rng.choice([0, 4, 5, 6, 7, 8]))
        dmax = digits or 8
        for fused in (True, False):
            p, d, w, s = raster.sort_plan_for(tiles, least, greatest, digits, fused)
            assert w == (greatest - least).bit_length()
            total = tile_bits(tiles) + w
            raw = min(max(-(-total // dmax), 2), 12)
            assert p == (raw if fused else raw + (raw & 1))
            assert d == -(-total // p) and d <= max(dmax, -(-total // 12)) and p * d >= total
            assert s == (p & 1 if fused else 0) and (fused or p % 2 == 0)


def test_image_keeps_key_order():
    """Sorting random keys of a frame by their images equals sorting the keys."""
    rng = np.random.default_rng(6)
    for _ in range(20):
        tiles = int(rng.integers(1, 5000))
        depth = rng.uniform(0.5, 200.0, 5000).astype(np.float32)
        bits = depth.view(np.uint32).astype(np.uint64)
        tile = rng.integers(0, tiles, 5000).astype(np.uint64)
        keys = (tile << np.uint64(32)) | bits
        least, greatest = int(bits.min()), int(bits.max())
        p, d, w, s = raster.sort_plan_for(tiles, least, greatest)
        image = (tile << np.uint64(w)) | (bits - np.uint64(least))
        assert int(image.max()) < (1 << (tile_bits(tiles) + w)) or tiles == 1
        assert np.array_equal(np.argsort(image, kind="stable"), np.argsort(keys, kind="stable"))
