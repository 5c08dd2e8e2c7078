"""Failure handling on the GPU, in the forms that fault and hang nothing.

* A sort look-back wait that runs out: with gs_set_sort_wait, one key
  partition of every pass withholds its digit counts (a flag nothing else
  sets), so its successor's bounded wait expires.  The frame must report
  GS_ERR_TIMEOUT, the later stages must see no keys (background image), and
  the context must render the next frame correctly.
* Non-finite parameters and zero quaternions mixed into a normal scene: culled
  exactly like the oracle culls them (same keys, ranges and image) and counted.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2412_00578_gb300 import synth

pytestmark = pytest.mark.gpu

BG = (0.1, 0.2, 0.3)


@pytest.fixture(scope="module")
def raster():
    from paper_2412_00578_gb300 import build

    build.build()
    from paper_2412_00578_gb300 import raster as r

    return r


def forward(raster, rast, scene_dev, cam, cfg, frame):
    rast.gs_preprocess(scene_dev, cam, cfg, frame)
    rast.gs_intersect(cam, cfg, frame)
    rast.gs_sort(cam, cfg, frame)
    rast.gs_tile_ranges(cam, cfg, frame)
    rast.gs_render(cam, cfg, frame)


def test_sort_wait_runs_out_then_context_recovers(raster):
    scene, cam = synth.small_box_workload()
    ref = oracle.render(scene, cam, 16, 2, bg=BG, prec64=False)
    K = ref["num_keys"]
    assert K > 3 * 4096  # partition 1 withholds, partition 2 waits on it
    rast = raster.Rasterizer("cuda:0")
    ds = scene.to("cuda:0")
    cfg = raster.cfg_struct(16, "accutile", BG)
    frame = raster.Frame(scene.n, cam.width, cam.height, 16, K + 100, "cuda:0")

    rast.gs_set_sort_wait(4096, 1)
    forward(raster, rast, ds, cam, cfg, frame)
    k, flags = rast.gs_read_status(frame, raise_on_error=False)
    assert flags & raster.FLAG_TIMEOUT and k == K
    with pytest.raises(raster.GsError) as ei:
        rast.gs_read_status(frame)
    assert ei.value.status == 5  # GS_ERR_TIMEOUT
    # after the expiry no stage reads the keys: empty ranges, background image
    assert int(frame.tile_ranges().abs().sum()) == 0
    img = frame.image.cpu().numpy()
    for c in range(3):
        assert np.all(img[c] == np.float32(BG[c]))
    assert int(frame.last.abs().sum()) == 0

    # normal waits again: the same context and frame render the oracle's frame
    rast.gs_set_sort_wait(0, -1)
    forward(raster, rast, ds, cam, cfg, frame)
    k, flags = rast.gs_read_status(frame)
    assert flags == 0 and k == K
    assert np.array_equal(frame.keys[:K].cpu().numpy().view(np.uint64), ref["keys"])
    assert np.array_equal(frame.vals[:K].cpu().numpy().view(np.uint32), ref["vals"])
    assert np.array_equal(frame.tile_ranges().cpu().numpy().view(np.uint32), ref["ranges"])
    assert np.abs(frame.image.cpu().numpy().astype(np.float64) - ref["image"]).max() <= 1e-4


def test_sort_rejects_keys_outside_the_recorded_range(raster):
    """gs_sort orders keys by (tile, depth bits - least depth bits) over the
    span gs_intersect recorded; a key changed after the emit to lie below that
    span is reported (GS_FLAG_KEYRANGE, GS_ERR_INVALID), the later stages see
    no keys, and the next frame renders normally."""
    scene, cam = synth.small_box_workload()
    ref = oracle.render(scene, cam, 16, 2, bg=BG, prec64=False)
    K = ref["num_keys"]
    rast = raster.Rasterizer("cuda:0")
    ds = scene.to("cuda:0")
    cfg = raster.cfg_struct(16, "accutile", BG)
    frame = raster.Frame(scene.n, cam.width, cam.height, 16, K + 100, "cuda:0")
    rast.gs_preprocess(ds, cam, cfg, frame)
    rast.gs_intersect(cam, cfg, frame)
    passes, _, w = rast.gs_read_sort_plan(cfg, frame)
    assert w < 32 and passes < 6
    torch.cuda.synchronize()
    keys = frame.keys[:K].view(torch.int64)
    keys[K // 2] = keys[K // 2] & ~0xFFFFFFFF  # depth bits 0: below every recorded depth
    torch.cuda.synchronize()
    rast.gs_sort(cam, cfg, frame)
    rast.gs_tile_ranges(cam, cfg, frame)
    rast.gs_render(cam, cfg, frame)
    k, flags = rast.gs_read_status(frame, raise_on_error=False)
    assert flags & raster.FLAG_KEYRANGE and k == K
    with pytest.raises(raster.GsError) as ei:
        rast.gs_read_status(frame)
    assert ei.value.status == 1  # GS_ERR_INVALID
    assert int(frame.tile_ranges().abs().sum()) == 0
    img = frame.image.cpu().numpy()
    for c in range(3):
        assert np.all(img[c] == np.float32(BG[c]))

    forward(raster, rast, ds, cam, cfg, frame)
    k, flags = rast.gs_read_status(frame)
    assert flags == 0 and k == K
    assert np.array_equal(frame.keys[:K].cpu().numpy().view(np.uint64), ref["keys"])
    assert np.array_equal(frame.vals[:K].cpu().numpy().view(np.uint32), ref["vals"])
    assert np.abs(frame.image.cpu().numpy().astype(np.float64) - ref["image"]).max() <= 1e-4


def poisoned_scene():
    scene = synth.uniform_box_scene(3000, seed=41, log_scale_mu=-3.0)
    nan, inf = float("nan"), float("inf")
    scene.means[0, 5] = nan
    scene.means[2, 50] = -inf
    scene.scales[1, 17] = inf
    scene.scales[0, 18] = nan
    scene.opacities[33] = nan
    scene.rotations[:, 71] = 0.0          # zero quaternion
    scene.rotations[2, 90] = nan
    scene.opacities[120] = inf
    # the definition of the culled set: any non-finite geometry or opacity
    # parameter, or a zero quaternion
    geo = np.concatenate([scene.means.numpy(), scene.scales.numpy(), scene.rotations.numpy(),
                          scene.opacities.numpy()[None]], 0)
    bad = ~np.isfinite(geo).all(0) | (np.abs(scene.rotations.numpy()).sum(0) == 0)
    return scene, int(bad.sum())


@pytest.mark.parametrize("mode", ["accutile", "3sigma"])
def test_non_finite_parameters_culled_and_counted(raster, mode):
    scene, n_bad = poisoned_scene()
    assert n_bad == 8
    cam = synth.pinhole(97, 61, 60.0, np.eye(3), np.array([0.0, 0.0, 5.0]))
    m = raster.MODES[mode]
    ref = oracle.render(scene, cam, 16, m, bg=BG, prec64=False)
    rast = raster.Rasterizer("cuda:0")
    frame = raster.Frame(scene.n, cam.width, cam.height, 16, 2 * ref["num_keys"] + 10, "cuda:0")
    cfg = raster.cfg_struct(16, mode, BG)
    forward(raster, rast, scene.to("cuda:0"), cam, cfg, frame)
    K, flags = rast.gs_read_status(frame)
    assert K == ref["num_keys"] and flags == 0
    counts = frame.counts[: scene.n].cpu().numpy()
    _, ocounts = oracle.preprocess(scene, cam, 16, m, prec64=False)
    assert np.array_equal(counts, ocounts)
    assert np.array_equal(frame.keys[:K].cpu().numpy().view(np.uint64), ref["keys"])
    assert np.array_equal(frame.vals[:K].cpu().numpy().view(np.uint32), ref["vals"])
    img = frame.image.cpu().numpy()
    assert np.isfinite(img).all()
    assert np.abs(img.astype(np.float64) - ref["image"]).max() <= 1e-4
    assert rast.gs_read_culled(frame) == n_bad
    # a clean frame afterwards counts none
    clean = synth.uniform_box_scene(3000, seed=41, log_scale_mu=-3.0)
    forward(raster, rast, clean.to("cuda:0"), cam, cfg, frame)
    rast.gs_read_status(frame)
    assert rast.gs_read_culled(frame) == 0
