"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: integer work (tile counts, key totals, emitted pairs, sorted pairs,
tile ranges, last-contributor indices) bit-exact against the FP32 oracle,
which follows the same documented operation order; the per-Gaussian 2D state
bit-exact; images within 1e-4 max abs error per channel (the FP64 oracle's
error is printed beside it).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2412_00578_gb300 import synth

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


@pytest.fixture(scope="module")
def raster():
    from paper_2412_00578_gb300 import build

    build.build()
    from paper_2412_00578_gb300 import raster as r

    return r


@pytest.fixture(scope="module")
def rast(raster):
    return raster.Rasterizer("cuda:0")


def expected_sort_plan(keys, tiles, sort_digit_bits):
    """The sort's plan for these keys: the tile bits, the bit length of the
    span of their depth bits (all 32 without keys), at most 8 (or the
    override's) bits per digit, 2 to 12 passes, digits as even as they go."""
    tile_bits = max(int(tiles) - 1, 0).bit_length()
    if len(keys):
        d = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
        w = int(d.max() - d.min()).bit_length()
    else:
        w = 32
    dmax = sort_digit_bits if 4 <= sort_digit_bits <= 8 else 8
    total = tile_bits + w
    passes = min(max(-(-total // dmax), 2), 12)
    return passes, -(-total // passes), w


def run_pipeline(raster, rast, scene, cam, mode, tile, bg=(0.0, 0.0, 0.0), n_capacity=None, key_capacity=None,
                 sort_digit_bits=0):
    """Run the five stages through the C ABI, snapshotting each stage's output."""
    dev_scene = scene.to("cuda:0")
    n = scene.n
    ncap = n if n_capacity is None else n_capacity
    if key_capacity is None:
        key_capacity = max(oracle.count_keys(scene, cam, tile, mode, prec64=False), 1)
    frame = raster.Frame(ncap, cam.width, cam.height, tile, key_capacity, "cuda:0")
    cfg = raster.cfg_struct(tile, mode, bg, sort_digit_bits)
    out = {}
    rast.gs_preprocess(dev_scene, cam, cfg, frame)
    torch.cuda.synchronize()
    out["counts"] = frame.counts[:ncap].cpu().numpy()
    out["proj"] = frame.proj_planes().cpu().numpy() if ncap > 0 else np.zeros((3, 0, 4), np.float32)
    K = rast.gs_intersect(cam, cfg, frame, sync=True)
    out["K"] = K
    Ke = min(K, key_capacity)
    out["keys_unsorted"] = frame.keys[:Ke].cpu().numpy().view(np.uint64).copy()
    out["vals_unsorted"] = frame.vals[:Ke].cpu().numpy().view(np.uint32).copy()
    if K <= key_capacity:
        # the sort keeps only the depth bits the emitted keys span
        tiles = -(-cam.width // tile) * -(-cam.height // tile)
        assert rast.gs_read_sort_plan(cfg, frame) == expected_sort_plan(out["keys_unsorted"], tiles, sort_digit_bits)
    rast.gs_sort(cam, cfg, frame)
    rast.gs_tile_ranges(cam, cfg, frame)
    rast.gs_render(cam, cfg, frame)
    torch.cuda.synchronize()
    out["keys"] = frame.keys[:Ke].cpu().numpy().view(np.uint64).copy()
    out["vals"] = frame.vals[:Ke].cpu().numpy().view(np.uint32).copy()
    out["ranges"] = frame.tile_ranges().cpu().numpy().view(np.uint32).copy()
    out["image"] = frame.image.cpu().numpy()
    out["final_T"] = frame.final_T.cpu().numpy()
    out["last"] = frame.last.cpu().numpy().view(np.uint32)
    out["frame"] = frame
    return out


def check_against_oracle(gpu, scene, cam, mode, tile, bg=(0.0, 0.0, 0.0), report_f64=False):
    ref = oracle.render(scene, cam, tile, mode, bg=bg, prec64=False)
    st, counts = oracle.preprocess(scene, cam, tile, mode, prec64=False)
    n = scene.n
    # counts and per-Gaussian 2D state
    assert np.array_equal(gpu["counts"][:n], counts), "tile counts differ"
    assert np.all(gpu["counts"][n:] == 0)
    m = counts > 0
    if m.any():
        P = gpu["proj"][:, :n]
        f32 = lambda a: a.astype(np.float32)
        np.testing.assert_array_equal(P[0][m], f32(st[m][:, [0, 1, 3, 2]]))  # u v opacity depth
        np.testing.assert_array_equal(P[1][m], f32(st[m][:, [4, 5, 6, 7]]))  # a b c t
        np.testing.assert_array_equal(P[2][m][:, :3], f32(st[m][:, [8, 9, 10]]))  # rgb
        assert np.array_equal(P[2][m][:, 3].view(np.int32), st[m][:, 14].astype(np.int32))  # radius
    # key total and emitted pairs (compared per Gaussian, any order within one)
    assert gpu["K"] == ref["num_keys"]
    ku, vu = gpu["keys_unsorted"], gpu["vals_unsorted"]
    o1 = np.lexsort((ku, vu))
    o2 = np.lexsort((ref["keys_unsorted"], ref["vals_unsorted"]))
    assert np.array_equal(vu[o1], ref["vals_unsorted"][o2]) and np.array_equal(ku[o1], ref["keys_unsorted"][o2])
    # emission is grouped by Gaussian in index order
    assert np.all(np.diff(vu.astype(np.int64)) >= 0)
    # sort, ranges: bit-exact
    assert np.array_equal(gpu["keys"], ref["keys"]), "sorted keys differ"
    assert np.array_equal(gpu["vals"], ref["vals"]), "sorted values differ"
    assert np.array_equal(gpu["ranges"], ref["ranges"]), "tile ranges differ"
    # image
    err = np.abs(gpu["image"].astype(np.float64) - ref["image"]).max() if gpu["image"].size else 0.0
    assert err <= IMG_TOL, err
    assert np.abs(gpu["final_T"].astype(np.float64) - ref["final_T"]).max() <= IMG_TOL
    assert np.array_equal(gpu["last"], ref["last"])
    if report_f64:
        ref64 = oracle.render(scene, cam, tile, mode, bg=bg, prec64=True)
        e64 = np.abs(gpu["image"].astype(np.float64) - ref64["image"]).max()
        print(f"mode {mode} tile {tile}: K={gpu['K']} max|gpu-f32 oracle|={err:.3g} max|gpu-f64 oracle|={e64:.3g}")
    return ref


def ragged_case(n=3000, seed=31, w=97, h=61):
    scene = synth.uniform_box_scene(n, seed=seed, log_scale_mu=-3.0)
    cam = synth.pinhole(w, h, 60.0, np.eye(3), np.array([0.0, 0.0, 5.0]))
    return scene, cam


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_ragged_small(raster, rast, mode, tile):
    scene, cam = ragged_case()
    gpu = run_pipeline(raster, rast, scene, cam, mode, tile, bg=(0.1, 0.2, 0.3))
    check_against_oracle(gpu, scene, cam, mode, tile, bg=(0.1, 0.2, 0.3))


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_render_stats_pair_counts(raster, rast, tile):
    """gs_render_stats: the evaluated and contributing pair counts (the blend
    work the benchmark's roofline divides by time) equal the oracle's walk;
    every contributing pair is among the pairs the kernel tested."""
    for scene, cam in [ragged_case(), synth.small_box_workload()]:
        gpu = run_pipeline(raster, rast, scene, cam, 2, tile)
        ev, co, ex = rast.gs_render_stats(cam, raster.cfg_struct(tile, 2), gpu["frame"])
        ref = oracle.render(scene, cam, tile, 2, prec64=False)
        assert ev == ref["evaluated_pairs"] and co == ref["contributing_pairs"]
        assert co <= ex


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
def test_box_16k_320x240(raster, rast, mode):
    scene, cam = synth.small_box_workload()
    gpu = run_pipeline(raster, rast, scene, cam, mode, 16)
    check_against_oracle(gpu, scene, cam, mode, 16, report_f64=True)


def test_orbit_camera_large_splats(raster, rast):
    """Off-axis camera, bigger Gaussians (many tiles each, both sweep
    directions, clipping at every image edge)."""
    scene = synth.uniform_box_scene(4000, seed=32, half=3.0, log_scale_mu=-2.0, log_scale_sd=0.7)
    cam = synth.look_at(211, 157, 60.0, (2.5, -1.5, -6.0), (0.3, 0.2, 0.1))
    for mode in (0, 1, 2, 3, 4):
        gpu = run_pipeline(raster, rast, scene, cam, mode, 16, bg=(0.5, 0.5, 0.5))
        check_against_oracle(gpu, scene, cam, mode, 16, bg=(0.5, 0.5, 0.5))


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_needles_and_faint_splats(raster, rast, tile):
    """Long thin splats at every orientation (conics from round to nearly
    singular) and faint ones (threshold t near 0, ellipses smaller than a
    pixel): the blend's per-warp culling must keep every pixel the per-pixel
    test accepts, so images and last-contributor indices stay bit-exact."""
    scene = synth.uniform_box_scene(6000, seed=41, half=2.0, log_scale_mu=-3.5, log_scale_sd=0.5)
    gen = torch.Generator().manual_seed(42)
    stretch = torch.exp(4.0 * torch.rand(6000, generator=gen))  # 1 .. 55 x
    scene.scales[0] *= stretch
    scene.scales[1] /= stretch
    faint = torch.rand(6000, generator=gen) < 0.3
    scene.opacities[faint] = 0.004 + 0.02 * torch.rand(int(faint.sum()), generator=gen)
    cam = synth.look_at(163, 119, 55.0, (0.7, -0.4, -5.5), (0.0, 0.0, 0.0))
    for mode in (2, 3, 4):
        gpu = run_pipeline(raster, rast, scene, cam, mode, tile, bg=(0.3, 0.1, 0.2))
        check_against_oracle(gpu, scene, cam, mode, tile, bg=(0.3, 0.1, 0.2))


def crowded_tile_case(n, seed):
    """n tiny Gaussians whose centres project inside tile (1, 1) of a 64x48
    image at tile 16 (pixels 16..31), half of them at one depth, so one
    bucket holds every key and depth ties are broken by Gaussian index."""
    scene = synth.uniform_box_scene(n, seed=seed, half=0.2, log_scale_mu=-7.0, log_scale_sd=0.3)
    scene.means[0] -= 0.9
    scene.means[1] += 0.06
    same = torch.arange(n) % 2 == 0
    scene.means[2, same] = 0.125
    cam = synth.pinhole(64, 48, 60.0, np.eye(3), np.array([0.0, 0.0, 5.0]))
    return scene, cam


@pytest.mark.parametrize("n", [6000, 40000])
def test_one_crowded_tile(raster, rast, n):
    """One tile holding 6000 or 40000 keys (a digit run far longer than a sort
    partition), half of them at one depth, so ties must keep Gaussian index
    order; keys, values, ranges and image as the oracle."""
    scene, cam = crowded_tile_case(n, seed=51)
    _, counts = oracle.preprocess(scene, cam, 16, 2, prec64=False)
    K = int(counts.sum())
    assert K > 0.99 * n and counts.max() == 1  # precondition: at most one tile per Gaussian
    gpu = run_pipeline(raster, rast, scene, cam, 2, 16)
    ref = check_against_oracle(gpu, scene, cam, 2, 16)
    r = ref["ranges"].reshape(-1, 2)
    assert r[1 * 4 + 1, 1] - r[1 * 4 + 1, 0] == K  # all of them in tile (1, 1)


def test_one_depth_for_the_whole_frame(raster, rast):
    """30,000 Gaussians on the plane z = 0 seen from z = 5: every key has the
    same depth bits, so each depth digit pass holds a single digit value (the
    sort's concentrated-digit ranking at its extreme) and every tile's order is
    Gaussian index order, decided by the sort's stability alone."""
    scene = synth.uniform_box_scene(30000, seed=61, half=2.0, log_scale_mu=-3.5, log_scale_sd=0.6)
    scene.means[2] = 0.0
    cam = synth.pinhole(320, 240, 60.0, np.eye(3), np.array([0.0, 0.0, 5.0]))
    gpu = run_pipeline(raster, rast, scene, cam, 2, 16)
    depth_bits = np.unique(gpu["keys_unsorted"] & np.uint64(0xFFFFFFFF))
    assert depth_bits.size == 1 and gpu["K"] > 30000  # precondition: one depth, many keys
    check_against_oracle(gpu, scene, cam, 2, 16)
    # within each tile the values ascend
    tiles = gpu["keys"] >> np.uint64(32)
    same = tiles[1:] == tiles[:-1]
    assert np.all(gpu["vals"][1:][same] > gpu["vals"][:-1][same])


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_one_depth_forward_keeps_no_depth_bits(raster, rast, tile):
    """The same one-depth frame through gs_forward: the plan keeps no depth
    bits (the tile bits alone decide the order, in two passes or more), and
    the pairs, ranges and image are the oracle's."""
    scene = synth.uniform_box_scene(30000, seed=61, half=2.0, log_scale_mu=-3.5, log_scale_sd=0.6)
    scene.means[2] = 0.0
    cam = synth.pinhole(320, 240, 60.0, np.eye(3), np.array([0.0, 0.0, 5.0]))
    frame, K = check_forward(raster, rast, scene, cam, 2, tile)
    passes, dbits, w = rast.gs_read_sort_plan(raster.cfg_struct(tile, 2), frame)
    tiles = -(-cam.width // tile) * -(-cam.height // tile)
    assert w == 0 and passes * dbits >= max(tiles - 1, 0).bit_length() and passes >= 2


@pytest.mark.parametrize("digits", [6, 5, 4])
def test_digit_widths_agree(raster, rast, digits):
    """Narrower radix digits (more passes) give the same sorted pairs, bit for
    bit, as the default 8-bit digits."""
    for scene, cam, mode in [(*ragged_case(), 0), (*crowded_tile_case(6000, seed=52), 2)]:
        a = run_pipeline(raster, rast, scene, cam, mode, 16)
        b = run_pipeline(raster, rast, scene, cam, mode, 16, sort_digit_bits=digits)
        for k in ("keys", "vals", "ranges", "image", "last"):
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_sh_degrees(raster, rast, deg):
    scene, cam = ragged_case(n=1500, seed=33)
    scene.sh_degree = deg
    gpu = run_pipeline(raster, rast, scene, cam, 2, 16)
    check_against_oracle(gpu, scene, cam, 2, 16)


def test_padding_capacity_beyond_n(raster, rast):
    scene, cam = ragged_case(n=1000, seed=34)
    gpu = run_pipeline(raster, rast, scene, cam, 2, 16, n_capacity=1000 + 4099)
    check_against_oracle(gpu, scene, cam, 2, 16)


def test_empty_scene_and_all_culled(raster, rast):
    _, cam = ragged_case()
    empty = synth.uniform_box_scene(0, seed=35)
    gpu = run_pipeline(raster, rast, empty, cam, 2, 16, bg=(0.2, 0.3, 0.4), key_capacity=16)
    assert gpu["K"] == 0
    assert np.allclose(gpu["image"], np.array([0.2, 0.3, 0.4], np.float32)[:, None, None])
    assert np.all(gpu["final_T"] == 1.0) and np.all(gpu["last"] == 0) and np.all(gpu["ranges"] == 0)
    behind = synth.uniform_box_scene(2000, seed=36)
    behind.means[2] -= 20.0  # all behind the camera
    gpu = run_pipeline(raster, rast, behind, cam, 2, 16, key_capacity=16)
    assert gpu["K"] == 0 and np.all(gpu["counts"] == 0)


def test_screen_filling_gaussian(raster, rast):
    """One large opaque Gaussian in front of the camera touches every tile."""
    scene = synth.uniform_box_scene(1, seed=37)
    scene.means[:] = torch.tensor([[0.0], [0.0], [-3.0]])
    scene.scales[:] = 5.0
    scene.opacities[:] = 0.99
    cam = synth.pinhole(100, 75, 60.0, np.eye(3), np.array([0.0, 0.0, 5.0]))
    for mode in (0, 1, 2):
        gpu = run_pipeline(raster, rast, scene, cam, mode, 16)
        assert gpu["K"] == 7 * 5
        check_against_oracle(gpu, scene, cam, mode, 16)


def test_capacity_overflow_reports_and_renderer_recovers(raster, rast):
    scene, cam = ragged_case(n=2000, seed=38)
    K = oracle.count_keys(scene, cam, 16, 2)
    frame = raster.Frame(scene.n, cam.width, cam.height, 16, K - 1, "cuda:0")
    cfg = raster.cfg_struct(16, 2)
    rast.gs_preprocess(scene.to("cuda:0"), cam, cfg, frame)
    assert rast.gs_intersect(cam, cfg, frame, sync=True) == K
    Kr, flags = rast.gs_read_status(frame, raise_on_error=False)
    assert Kr == K and flags & raster.FLAG_CAPACITY
    with pytest.raises(raster.GsError) as ei:
        rast.gs_read_status(frame)
    assert ei.value.status == 3
    r = raster.Renderer("cuda:0")
    r.frames[(scene.n, cam.width, cam.height, 16)] = raster.Frame(scene.n, cam.width, cam.height, 16, 100, "cuda:0")
    out = r.render(scene.to("cuda:0"), cam, "accutile", 16)
    ref = oracle.render(scene, cam, 16, 2, prec64=False)
    assert out.num_keys == K
    assert np.abs(out.image.cpu().numpy() - ref["image"]).max() <= IMG_TOL


def test_invalid_arguments_are_rejected(raster, rast):
    scene, cam = ragged_case(n=10, seed=39)
    frame = raster.Frame(10, cam.width, cam.height, 16, 64, "cuda:0")
    ds = scene.to("cuda:0")
    with pytest.raises(raster.GsError) as ei:
        rast.gs_preprocess(ds, cam, raster.cfg_struct(8, 2), frame)  # tile mismatch
    assert ei.value.status == 1
    with pytest.raises(raster.GsError):
        rast.gs_preprocess(ds, cam, raster.cfg_struct(16, 7), frame)  # bad mode
    other = synth.pinhole(50, 50, 60.0, np.eye(3), np.zeros(3))
    with pytest.raises(raster.GsError):
        rast.gs_render(other, raster.cfg_struct(16, 2), frame)  # camera/frame size mismatch
    big = synth.uniform_box_scene(11, seed=40).to("cuda:0")
    with pytest.raises(raster.GsError):
        rast.gs_preprocess(big, cam, raster.cfg_struct(16, 2), frame)  # n > n_capacity


def test_repeatable_bit_for_bit(raster, rast):
    scene, cam = synth.small_box_workload()
    a = run_pipeline(raster, rast, scene, cam, 2, 16)
    b = run_pipeline(raster, rast, scene, cam, 2, 16)
    for k in ("keys", "vals", "ranges", "image", "last"):
        assert np.array_equal(a[k], b[k]), k


# ---------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def outdoor():
    return synth.outdoor_workload()


@pytest.mark.parametrize("mode", [2, 1, 0, 3, 4])
def test_outdoor_3m_1280x840_full_frame(raster, outdoor, mode):
    """The 3M-Gaussian 1280x840 workload in the launch configuration the
    benchmark times (gs_forward, tile 16): every key, range and pixel."""
    scene, cam = outdoor
    r = raster.Renderer("cuda:0")
    ds = scene.to("cuda:0")
    out = r.render(ds, cam, mode=mode, tile=16)  # sizes the frame (stage calls)
    f = out.frame
    f.image.fill_(-1.0)
    f.keys.fill_(-1)
    r.rast.gs_forward(ds, cam, raster.cfg_struct(16, mode), f)  # the call the benchmark times
    K, flags = r.rast.gs_read_status(f)
    ref = oracle.render(scene, cam, 16, mode, prec64=False, omp=True)
    assert K == ref["num_keys"] and flags == 0
    assert np.array_equal(f.keys[:K].cpu().numpy().view(np.uint64), ref["keys"])
    assert np.array_equal(f.vals[:K].cpu().numpy().view(np.uint32), ref["vals"])
    assert np.array_equal(f.tile_ranges().cpu().numpy().view(np.uint32), ref["ranges"])
    err = np.abs(f.image.cpu().numpy().astype(np.float64) - ref["image"]).max()
    assert err <= IMG_TOL, err
    assert np.array_equal(f.last.cpu().numpy().view(np.uint32), ref["last"])
    print(f"outdoor 3M mode {mode}: K={K}, image max abs err {err:.3g}")


def test_4k_tile8_many_tiles():
    """3840x2160 at tile 8: 129,600 tiles, so 49-bit keys (an eight-pass sort of
    7-bit digits) and more tiles than the blend's launch-order table holds
    (tiles then run in index order); 400k blob Gaussians through the stage calls."""
    from paper_2412_00578_gb300 import raster

    scene = synth.blob_scene(400_000, seed=9)
    cam = synth.pinhole(3840, 2160, 60.0, np.eye(3), np.array([0.0, 0.0, 25.0]))
    ref = oracle.render(scene, cam, 8, 2, prec64=False)
    r = raster.Renderer("cuda:0")
    out = r.render(scene.to("cuda:0"), cam, mode="accutile", tile=8)
    torch.cuda.synchronize()
    K = out.num_keys
    assert K == ref["num_keys"] and ref["grid"][0] * ref["grid"][1] == 129_600
    assert np.array_equal(out.frame.keys[:K].cpu().numpy().view(np.uint64), ref["keys"])
    assert np.array_equal(out.frame.vals[:K].cpu().numpy().view(np.uint32), ref["vals"])
    assert np.array_equal(out.frame.tile_ranges().cpu().numpy().view(np.uint32), ref["ranges"])
    assert np.abs(out.image.cpu().numpy().astype(np.float64) - ref["image"]).max() <= IMG_TOL
    assert np.array_equal(out.last.cpu().numpy().view(np.uint32), ref["last"])


def test_outdoor_pruned_300k(raster, outdoor):
    scene, cam = outdoor
    pruned = synth.prune_random(scene, 300_000, seed=1)
    r = raster.Renderer("cuda:0")
    out = r.render(pruned.to("cuda:0"), cam, mode="accutile", tile=16)
    torch.cuda.synchronize()
    ref = oracle.render(pruned, cam, 16, 2, prec64=False)
    assert out.num_keys == ref["num_keys"]
    assert np.array_equal(out.frame.keys[:out.num_keys].cpu().numpy().view(np.uint64), ref["keys"])
    assert np.abs(out.image.cpu().numpy().astype(np.float64) - ref["image"]).max() <= IMG_TOL


def test_outdoor_10m_1920x1080_forward(raster):
    """A 10M-Gaussian scene of the same recipe at 1920x1080 (8,160 tiles,
    40,000 preprocess warps, over 2,400 scan blocks): the gs_forward chain with
    its device-chosen sort plan, against the oracle's keys, ranges and image."""
    scene, cam = synth.outdoor_workload(n=10_000_000, seed=4, width=1920, height=1080)
    r = raster.Rasterizer("cuda:0")
    ref = oracle.render(scene, cam, 16, 2, prec64=False, omp=True)
    K = ref["num_keys"]
    frame = raster.Frame(scene.n, cam.width, cam.height, 16, K + 1000, "cuda:0")
    cfg = raster.cfg_struct(16, 2)
    r.gs_forward(scene.to("cuda:0"), cam, cfg, frame)
    k, flags = r.gs_read_status(frame)
    assert k == K and flags == 0
    keys = ref["keys"]
    tiles = -(-cam.width // 16) * -(-cam.height // 16)
    assert r.gs_read_sort_plan(cfg, frame) == expected_sort_plan(keys, tiles, 0)
    assert np.array_equal(frame.keys[:K].cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(frame.vals[:K].cpu().numpy().view(np.uint32), ref["vals"])
    assert np.array_equal(frame.tile_ranges().cpu().numpy().view(np.uint32), ref["ranges"])
    assert np.abs(frame.image.cpu().numpy().astype(np.float64) - ref["image"]).max() <= IMG_TOL
    print(f"outdoor 10M 1920x1080: K={K}, plan {r.gs_read_sort_plan(cfg, frame)}")


# ---------------------------------------------------------------- gs_forward
def run_forward(raster, rast, scene, cam, mode, tile, bg=(0.0, 0.0, 0.0), key_capacity=None, n_capacity=None,
                sort_digit_bits=0):
    """gs_forward: the five stages in one call, launched as one chain."""
    ncap = scene.n if n_capacity is None else n_capacity
    if key_capacity is None:
        key_capacity = max(oracle.count_keys(scene, cam, tile, mode, prec64=False), 1)
    frame = raster.Frame(ncap, cam.width, cam.height, tile, key_capacity, "cuda:0")
    cfg = raster.cfg_struct(tile, mode, bg, sort_digit_bits)
    rast.gs_forward(scene.to("cuda:0"), cam, cfg, frame)
    K, flags = rast.gs_read_status(frame, raise_on_error=False)
    return frame, K, flags


def check_forward(raster, rast, scene, cam, mode, tile, bg=(0.0, 0.0, 0.0), **kw):
    frame, K, flags = run_forward(raster, rast, scene, cam, mode, tile, bg, **kw)
    ref = oracle.render(scene, cam, tile, mode, bg=bg, prec64=False)
    st, counts = oracle.preprocess(scene, cam, tile, mode, prec64=False)
    assert flags == 0 and K == ref["num_keys"]
    n = scene.n
    assert np.array_equal(frame.counts[:n].cpu().numpy(), counts)
    m = counts > 0
    if m.any():
        P = frame.proj_planes().cpu().numpy()[:, :n]
        f32 = lambda a: a.astype(np.float32)
        np.testing.assert_array_equal(P[0][m], f32(st[m][:, [0, 1, 3, 2]]))
        np.testing.assert_array_equal(P[1][m], f32(st[m][:, [4, 5, 6, 7]]))
        np.testing.assert_array_equal(P[2][m][:, :3], f32(st[m][:, [8, 9, 10]]))
    assert np.array_equal(frame.keys[:K].cpu().numpy().view(np.uint64), ref["keys"])
    assert np.array_equal(frame.vals[:K].cpu().numpy().view(np.uint32), ref["vals"])
    assert np.array_equal(frame.tile_ranges().cpu().numpy().view(np.uint32), ref["ranges"])
    assert np.abs(frame.image.cpu().numpy().astype(np.float64) - ref["image"]).max() <= IMG_TOL
    assert np.array_equal(frame.last.cpu().numpy().view(np.uint32), ref["last"])
    return frame, K


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_forward_ragged(raster, rast, mode, tile):
    scene, cam = ragged_case()
    check_forward(raster, rast, scene, cam, mode, tile, bg=(0.1, 0.2, 0.3))


@pytest.mark.parametrize("digits", [0, 7, 6, 5, 4])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_forward_sort_plans(raster, rast, digits, tile):
    """gs_forward's sort plan, chosen on the device from the recorded depth
    range, at every digit width: odd pass counts (the emit writes buffer 1 so
    the last pass ends in buffer 0) and even ones give the oracle's sorted
    pairs, ranges and image, and the plan is the one the keys imply."""
    scene, cam = synth.small_box_workload()
    frame, K = check_forward(raster, rast, scene, cam, 2, tile, sort_digit_bits=digits)
    cfg = raster.cfg_struct(tile, 2, (0.0, 0.0, 0.0), digits)
    keys = oracle.render(scene, cam, tile, 2, prec64=False)["keys"]
    tiles = -(-cam.width // tile) * -(-cam.height // tile)
    assert rast.gs_read_sort_plan(cfg, frame) == expected_sort_plan(keys, tiles, digits)


def test_forward_sort_plans_cover_both_parities():
    """The plans of test_forward_sort_plans include odd and even pass counts."""
    scene, cam = synth.small_box_workload()
    parities = set()
    for tile in (8, 16, 32):
        keys = oracle.render(scene, cam, tile, 2, prec64=False)["keys"]
        tiles = -(-cam.width // tile) * -(-cam.height // tile)
        for digits in (0, 7, 6, 5, 4):
            parities.add(expected_sort_plan(keys, tiles, digits)[0] % 2)
    assert parities == {0, 1}


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
def test_forward_many_blocks(raster, rast, mode):
    """The 16k box (16 scan blocks, 9 sort partitions) and a capacity padded
    past n (scan blocks with no Gaussians)."""
    scene, cam = synth.small_box_workload()
    check_forward(raster, rast, scene, cam, mode, 16)
    check_forward(raster, rast, scene, cam, mode, 16, n_capacity=scene.n + 5000)


def test_forward_large_splats_and_empty(raster, rast):
    scene, cam = synth.small_box_workload(seed=3)
    scene.scales = scene.scales * 8.0  # many multi-line AccuTile sets
    for mode in (0, 1, 2):
        check_forward(raster, rast, scene, cam, mode, 16)
    empty = synth.uniform_box_scene(0, seed=1)
    frame, K, flags = run_forward(raster, rast, empty, cam, 2, 16, bg=(0.2, 0.3, 0.4), key_capacity=16)
    assert K == 0 and flags == 0
    assert np.all(frame.image.cpu().numpy()[0] == np.float32(0.2))


def test_forward_capacity_one_short(raster, rast):
    scene, cam = synth.small_box_workload(seed=5)
    K = oracle.count_keys(scene, cam, 16, 2)
    frame, Kr, flags = run_forward(raster, rast, scene, cam, 2, 16, key_capacity=K - 1)
    assert Kr == K and flags & raster.FLAG_CAPACITY
    # nothing was sorted, ranged or blended: empty ranges, background
    assert int(frame.tile_ranges().abs().sum()) == 0
    assert float(frame.image.abs().max()) == 0.0
    # the same frame buffers at capacity K render the oracle's frame
    check_forward(raster, rast, scene, cam, 2, 16, key_capacity=K)
