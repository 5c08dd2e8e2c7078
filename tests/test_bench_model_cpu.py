"""The benchmark's algorithmic byte model per stage (what each stage must move
at the least, from the data layout: 236-byte Gaussians in planar SoA, a 4-byte
count each, three 16-byte planes of 2D state per counted Gaussian, 12-byte
(key, value) pairs, 8-byte tile ranges, a 20-byte pixel record), checked one
unit at a time so the roofline fractions divide by the stated figures."""
import bench

SH3 = 4 * 3 * 16  # degree-3 SH coefficients per Gaussian, bytes


def work(n=0, n_counted=0, keys=0, pixels=0, tiles=0, passes=5):
    return bench.stage_work(None, n, n_counted, keys, SH3, pixels, tiles, passes)


def test_per_gaussian():
    w = work(n=1)
    assert w["preprocess"] == 12 + 12 + 16 + 4 + 4  # mean, scale, rotation, opacity read; count written
    assert w["intersect"] == 4 + 4  # the count, read by the scan and by the emit
    assert w["sort"] == w["tile_ranges"] == w["render"] == 0


def test_per_counted_gaussian():
    w = work(n_counted=1)
    assert w["preprocess"] == SH3 + 3 * 16  # SH read, 2D state written
    assert w["intersect"] == 2 * 16  # the two planes the tile function reads
    assert w["render"] == 3 * 16  # the 2D state gathered once


def test_per_key_pixel_tile():
    w = work(keys=1)
    assert w["intersect"] == 8 + 4  # (key, value) written
    assert w["sort"] == 2 * (8 + 4)  # read and written once
    assert w["sort_design"] == 8 + 5 * 2 * (8 + 4)  # one histogram read + one read and write per pass
    assert w["tile_ranges"] == 8
    assert w["render"] == 4  # the value (Gaussian index)
    assert work(pixels=1)["render"] == 3 * 4 + 4 + 4  # RGB, final T, last index
    assert work(tiles=1)["tile_ranges"] == 8
